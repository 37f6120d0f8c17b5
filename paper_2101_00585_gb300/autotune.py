"""Tile autotuner for the batched registration launch.

Times every candidate (threads per CTA, keyframe chunk) on the actual batch
with CUDA events, keeps the fastest, and caches the choice in a JSON file keyed
by the GPU name and the batch shape (keyframe sizes, hypotheses per keyframe).
"""
from __future__ import annotations

import json
import os

import torch

CANDIDATES = ((256, 256), (256, 512), (512, 512), (512, 1024), (512, 2048))
CACHE = os.environ.get("UPSLAM_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "upslam_gb300", "batch_tiles.json"))


def shape_key(batch) -> str:
    sizes = ",".join(f"{k.pp.rows}x{k.pp.cols}" for k in batch.kfs)
    return f"{torch.cuda.get_device_name()}|sweep{batch.sw.pp.rows}x{batch.sw.pp.cols}|hyp{batch.n_hyp}|{sizes}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(batch, init_poses: torch.Tensor, params, reps: int = 3, use_cache: bool = True) -> dict:
    """Pick the fastest tiles for ``batch``; returns {"tiles": (threads, chunk), "ms": {...}, "cached": bool}."""
    key = shape_key(batch)
    cache = _load() if use_cache else {}
    if key in cache:
        batch.set_tiles(tuple(cache[key]["tiles"]))
        return {"tiles": tuple(cache[key]["tiles"]), "ms": cache[key]["ms"], "cached": True}
    times = {}
    for cand in CANDIDATES:
        batch.set_tiles(cand)
        batch.run(init_poses, params)  # warm-up
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            batch.run(init_poses, params)
            b.record()
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        times[f"{cand[0]}x{cand[1]}"] = best
    pick = min(CANDIDATES, key=lambda c: times[f"{c[0]}x{c[1]}"])
    batch.set_tiles(pick)
    if use_cache:
        cache[key] = {"tiles": list(pick), "ms": times}
        try:
            os.makedirs(os.path.dirname(CACHE), exist_ok=True)
            with open(CACHE, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return {"tiles": pick, "ms": times, "cached": False}
