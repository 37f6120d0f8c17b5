"""The benchmark's reference arm on CPU: the FP64 oracle timed on the host, one JSON line.

Checks the line's contract (metric, unit and direction shared with the GPU arm; the CPU
baseline and e2e objects) and that ranks other than 0 exit cleanly without work.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    import bench
    r = _run()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["workload"].startswith("tunnel 64x1024 sweeps vs 512x2048")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    r = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_training_step_bytes_count_each_tensor_use():
    """The training step's compulsory traffic, counted tensor by tensor for batch 1 (BF16, 2 bytes):
    x0 = 64*256*8, layer outputs a0..a3 = 32*128*32, 16*64*64, 8*32*128, 4*16*128 elements."""
    import bench
    x0, a = 64 * 256 * 8, [32 * 128 * 32, 16 * 64 * 64, 8 * 32 * 128, 4 * 16 * 128]
    forward = x0 + 2 * sum(a)                       # read x0; each output written, then read once
    weight_grads = (x0 + a[0]) + (a[0] + a[1]) + (a[1] + a[2]) + (a[2] + a[3])
    data_grads = sum(a[l] + 2 * a[l - 1] for l in (1, 2, 3))  # read dY and the mask, write the dY below
    gather = 2 * x0
    elems = forward + a[3] + weight_grads + data_grads + gather  # + the last dY, written by the head
    assert bench.cnn_step_bytes(1) == 2 * elems
    assert bench.cnn_step_bytes(256) == 256 * bench.cnn_step_bytes(1)
