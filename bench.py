#!/usr/bin/env python
"""Throughput of the UPSLAM per-sweep hot path on GB300.

Workload (the headline configuration): 64 x 1024 lidar sweeps (FOV +-16.6 deg,
range 0.5-120 m, sigma 2 cm, 2 % dropouts) along a seeded 200 m trajectory
through a procedural tunnel / corridor network; keyframe panoramas 512 x 2048
with FP32 depth, FP32 normals and FP32 sample counts; a new keyframe every 5 m.
One step = one sweep through the whole path in one persistent launch: projection
+ z-buffer, normals, motion prior, ICP (up to 15 Gauss-Newton steps) and the
keyframe update (plus a new keyframe every 50 sweeps).

Metric: sweeps per second (ICP + fusion scans/s at 64 x 1024).  Inputs are
resident in HBM when the timed region starts; the timed steps run as one CUDA
graph with event-record nodes around every step and around the ICP and fusion
launches; L2 is flushed (a 256 MiB write) between steps, outside the events.
``e2e`` repeats the measurement through the public API from pinned host memory
(host->device copy of each sweep, device->host read of its pose and record,
one synchronisation per sweep).  ``cpu_baseline`` times the FP64 oracle on the
host cores on a bounded sample of the same sweeps.

``--impl reference`` times the oracle (the only reference there is) on the host
cores, rank 0 only, on a bounded sample sized to finish in a few minutes.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ICP+fusion scans/s at 64x1024"
UNIT = "scans/s"
KF_ROWS, KF_COLS = 512, 2048
FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0
LEARNED_ICP_STEPS = 12
DIFF_TIMING = ("difference of two graph replays, 20 calls each with and without the timed call "
               "(inputs restored and L2 flushed before every call), CUDA events around each replay")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["tunnel", "room", "campus", "forest-batch", "learned"], default="tunnel",
                    help="tunnel: the headline line; campus: the FP16 precision form; forest-batch: the batched "
                         "form; learned: train the pose proposal and evaluate learned vs plain initialisation")
    ap.add_argument("--train-pairs", type=int, default=200000)
    ap.add_argument("--eval-pairs", type=int, default=5000)
    ap.add_argument("--epochs", type=int, default=24)
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-graph", action="store_true", help="launch eagerly instead of replaying a CUDA graph")
    ap.add_argument("--atrous-levels", type=int, default=3,
                    help="also time the a-trous normal smoothing with this many levels (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", choices=["all", "none"], default="all",
                    help="also run the other workloads (room latency, campus precision form, forest batched form, "
                         "learned proposal) after the headline and report them under 'forms'")
    ap.add_argument("--form-steps", type=int, default=40, help="timed sweeps of the campus form")
    ap.add_argument("--batch-keyframes", type=int, default=64,
                    help="forest batched form: keyframes in the batch (the workload has 64; fewer for profiling)")
    ap.add_argument("--no-autotune", action="store_true", help="forest batched form: default tiles (512 x 512)")
    ap.add_argument("--quiet", action="store_true")
    return ap.parse_args()


def log(msg):
    sys.stderr.write(msg + "\n")
    sys.stderr.flush()


# ----------------------------------------------------------------------------- distributed plumbing

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
        return dist
    return None


def combine_ranks(local_ms: float, dist, device="cpu") -> float:
    """Timed duration of the whole job: the maximum over ranks (replicas run independently)."""
    if dist is None:
        return local_ms
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(steps: int, world: int, total_ms: float) -> float:
    """Whole-job throughput: every rank's sweeps over the slowest rank's time."""
    return world * steps / (total_ms * 1e-3)


# ----------------------------------------------------------------------------- workload

def make_workload(n_scans: int, rank: int = 0):
    from synth import configs
    seq = configs.tunnel_sequence(n_scans=max(n_scans, 2))
    t0 = time.time()
    scans = np.stack([seq.scan(k) for k in range(n_scans)])
    log(f"[bench] rank {rank}: generated {n_scans} sweeps of {scans.shape[1]} points in {time.time() - t0:.1f} s")
    return seq, scans


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                d = json.load(f)
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in d:
                    v = d[key]
                    if isinstance(v, dict):
                        v = v.get("value", v.get("burst"))
                    return float(v), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


FALLBACK_BF16_TFLOPS = {"burst": 1900.0, "sustained": 1700.0}


def bf16_peak(kind: str = "sustained"):
    """Dense BF16 tensor throughput (TFLOP/s) from MEASURED_PEAKS.json: the burst figure for a kernel timed
    alone, the sustained one for work timed inside a long loop; else the fallback figures."""
    key = "bf16_tflops_sustained" if kind == "sustained" else "bf16_tflops"
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = json.load(f).get(key)
        if v:
            return float(v), f"measured {kind}"
    except (OSError, ValueError):
        pass
    return FALLBACK_BF16_TFLOPS[kind], f"fallback {kind}"


PROFILE = os.path.join(ROOT, "profiles", "icp_tile_kernel_tunnel_64x1024_kf512x2048.md")
PROFILED_SOURCES = ("paper_2101_00585_gb300/csrc/icp.cu", "paper_2101_00585_gb300/csrc/common.cuh", "include/upslam.h")


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary, or None once the kernel sources changed."""
    import hashlib
    try:
        txt = open(PROFILE).read()
        h = hashlib.sha256()
        for f in PROFILED_SOURCES:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
        if f"source_sha256: {h.hexdigest()}" not in txt:
            return None
        for line in txt.splitlines():
            if line.startswith("| traffic_bytes_per_launch |"):
                return int(line.split("|")[2].strip())
    except OSError:
        return None
    return None


# ----------------------------------------------------------------------------- CUDA events usable inside graphs

class Cudart:
    """cudaEventRecordWithFlags(..., cudaEventRecordExternal) so events become graph nodes."""

    def __init__(self):
        lib = None
        for name in ("libcudart.so.13", "libcudart.so.12", "libcudart.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if lib is None:
            raise RuntimeError("libcudart not found")
        self.lib = lib
        lib.cudaEventCreate.argtypes = [ctypes.POINTER(ctypes.c_void_p)]
        lib.cudaEventRecordWithFlags.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint]
        lib.cudaEventElapsedTime.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_void_p, ctypes.c_void_p]
        lib.cudaEventSynchronize.argtypes = [ctypes.c_void_p]
        lib.cudaEventDestroy.argtypes = [ctypes.c_void_p]

    def event(self):
        ev = ctypes.c_void_p()
        assert self.lib.cudaEventCreate(ctypes.byref(ev)) == 0
        return ev

    # events become graph nodes only while a stream is being captured; eager launches record plainly
    external = True

    def record(self, ev, stream):
        rc = self.lib.cudaEventRecordWithFlags(ev, ctypes.c_void_p(stream), 1 if self.external else 0)
        assert rc == 0, rc

    def elapsed(self, a, b) -> float:
        ms = ctypes.c_float()
        assert self.lib.cudaEventSynchronize(b) == 0
        assert self.lib.cudaEventElapsedTime(ctypes.byref(ms), a, b) == 0
        return ms.value


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- our arm

def run_ours(args, ws, rank, local):
    import torch
    import paper_2101_00585_gb300 as up

    torch.cuda.set_device(local)
    dist = init_dist(ws, "nccl")
    device = torch.device("cuda", local)
    W, K = args.warmup, args.steps
    n_scans = 1 + W + K
    seq, scans = make_workload(n_scans, rank)
    p = up.Params(accept_quality=0.1)
    trk = up.Tracker(seq.sweep, seq.kf, p, device=device, constant_velocity=True)
    kf_every = seq.kf_every
    # keyframe pool: every keyframe the sequence will start, zeroed up front
    n_kf = 2 + n_scans // kf_every
    pool = [trk.kf] + [up.KeyframeBuffer(seq.kf, device) for _ in range(n_kf)]
    pool_pos = [0]
    h_scans = torch.from_numpy(scans).pin_memory()
    d_scans = h_scans.to(device)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    hist_pose = torch.zeros((n_scans, 12), dtype=torch.float64, device=device)
    hist_stats = torch.zeros((n_scans, up._abi.STATS_BYTES), dtype=torch.uint8, device=device)
    switched_after = []

    def switch_keyframe():
        pool_pos[0] += 1
        trk.new_keyframe(buffer=pool[pool_pos[0]])

    def step(k):
        trk.track(d_scans[k])
        if k % kf_every == 0:
            switch_keyframe()
            switched_after.append(k)

    torch.cuda.synchronize()
    # sweep 0 opens the first keyframe; warm-up sweeps 1..W run eagerly
    trk.new_keyframe(d_scans[0])
    for k in range(1, 1 + W):
        step(k)
        hist_pose[k].copy_(trk.state.pose)
        hist_stats[k].copy_(trk.state.stats)
    torch.cuda.synchronize()

    cr = Cudart()
    s = torch.cuda.Stream(device)
    ev = [(cr.event(), cr.event()) for _ in range(K)]
    ev_icp = [(cr.event(), cr.event()) for _ in range(K)]
    ev_fuse = [(cr.event(), cr.event()) for _ in range(K)]
    ev_proj = [(cr.event(), cr.event()) for _ in range(K)]
    trk.timing = None
    launches = [0]

    def timed_steps():
        st = torch.cuda.current_stream().cuda_stream
        for i in range(K):
            k = 1 + W + i
            trk.timing = (cr, st, ev_proj[i], ev_icp[i], ev_fuse[i])
            cr.record(ev[i][0], st)
            step(k)
            cr.record(ev[i][1], st)
            launches[0] += trk.launches_per_track + (up.Tracker.LAUNCHES_PER_NEW_KEYFRAME
                                                     if k % kf_every == 0 else 0)
            hist_pose[k].copy_(trk.state.pose)
            hist_stats[k].copy_(trk.state.stats)
            flush.zero_()
        trk.timing = None

    used_graph = False
    with torch.cuda.stream(s):
        if not args.no_graph:
            try:
                g = torch.cuda.CUDAGraph()
                saved = (pool_pos[0], list(switched_after))
                with torch.cuda.graph(g, stream=s):
                    timed_steps()
                pool_pos[0], switched_after[:] = saved[0], saved[1]
                used_graph = True
            except Exception as e:  # capture unsupported: launch eagerly
                log(f"[bench] graph capture failed ({e}); launching eagerly")
                torch.cuda.synchronize()
                launches[0] = 0
        cr.external = used_graph
        sampler = ClockSampler(local)
        sampler.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        if used_graph:
            g.replay()
        else:
            timed_steps()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        clocks = sampler.stop()
    step_ms = [cr.elapsed(a, b) for a, b in ev]
    icp_ms = [cr.elapsed(a, b) for a, b in ev_icp]
    fuse_ms = [cr.elapsed(a, b) for a, b in ev_fuse]
    proj_ms = [cr.elapsed(a, b) for a, b in ev_proj]
    total_ms = combine_ranks(float(sum(step_ms)), dist, device)

    # accuracy of the timed trajectory (host-side, after the fact)
    from paper_2101_00585_gb300._abi import IcpStats
    poses = hist_pose.cpu().numpy().reshape(-1, 3, 4)
    stats_raw = hist_stats.cpu().numpy()
    recs = [IcpStats.from_buffer_copy(bytes(stats_raw[k])) for k in range(n_scans)]
    iters = [recs[1 + W + i].iters for i in range(K)]
    accepted = sum(recs[1 + W + i].accepted for i in range(K))
    import synth
    P_kf = seq.poses[0]
    errs = []
    for k in range(1, n_scans):
        Pw = synth.pose_mul(P_kf, poses[k])
        errs.append(synth.pose_error(Pw, seq.poses[k]))
        if k % kf_every == 0:
            P_kf = Pw

    hbm, hbm_src = peaks()
    kf_px, sw_px = KF_ROWS * KF_COLS, seq.sweep.pixels
    icp_avg, fuse_avg, proj_avg = (statistics.mean(icp_ms), statistics.mean(fuse_ms), statistics.mean(proj_ms))
    if trk.front_fused:
        # one persistent launch per sweep.  Algorithmic bytes, the per-unit figures for this
        # workload: projection (the points, 16 B; the z-buffer touched twice and the outputs, 24 B per sweep
        # pixel: 2.6 MB), normals (32 B per sweep pixel: 2.1 MB), each Gauss-Newton step's correspondences
        # (48 B per sweep pixel: 3.1 MB per step, times the steps run), the keyframe read and written once
        # (40 B per keyframe pixel: 42 MB) and the hole fill's read of the sweep (24 B per sweep pixel)
        iters_mean = statistics.mean(iters)
        track_bytes = sw_px * (16 + 24) + sw_px * 32 + sw_px * 48 * iters_mean + kf_px * 40 + sw_px * 24
        # the same launch counted by what it touches once (the sweep read once by all steps)
        touched = kf_px * 40 + sw_px * 32 + sw_px * (16 + 24 + 40 + 20)
        name = "icp_tile_kernel (project + normals + register + keyframe update)"
        kernels = {name: {"ms_avg": icp_avg, "share": sum(icp_ms) / total_ms, "bytes": round(track_bytes),
                          "bytes_touched_once": touched, "gbs": track_bytes / (icp_avg * 1e-3) / 1e9,
                          "iters_avg": iters_mean}}
        dom = name
    elif trk.fused:
        # one persistent launch: ICP + keyframe update; the keyframe must be read once and written
        # once (20 B/px each way) and the sweep read once (32 B/px)
        track_bytes = kf_px * 40 + sw_px * 32
        kernels = {
            "icp_tile_kernel (register + keyframe update)": {
                "ms_avg": icp_avg, "share": sum(icp_ms) / total_ms, "bytes": track_bytes,
                "gbs": track_bytes / (icp_avg * 1e-3) / 1e9, "iters_avg": statistics.mean(iters)},
            "project + resolve + normals": {"ms_avg": proj_avg, "share": sum(proj_ms) / total_ms,
                                            "bytes": sw_px * (16 + 8 + 8 + 4 + 4 + 16 + 36),
                                            "gbs": sw_px * 92 / (proj_avg * 1e-3) / 1e9},
        }
        dom = "icp_tile_kernel (register + keyframe update)"
    else:
        icp_bytes = kf_px * 20 + sw_px * 32
        fuse_bytes = kf_px * 40 + sw_px * 32 * 2
        kernels = {
            "icp_tile_kernel": {"ms_avg": icp_avg, "share": sum(icp_ms) / total_ms, "bytes": icp_bytes,
                                "gbs": icp_bytes / (icp_avg * 1e-3) / 1e9, "iters_avg": statistics.mean(iters)},
            "fuse_main + fuse_fill": {"ms_avg": fuse_avg, "share": sum(fuse_ms) / total_ms, "bytes": fuse_bytes,
                                      "gbs": fuse_bytes / (fuse_avg * 1e-3) / 1e9},
            "project + resolve + normals": {"ms_avg": proj_avg, "share": sum(proj_ms) / total_ms},
        }
        dom = "icp_tile_kernel" if sum(icp_ms) >= sum(fuse_ms) else "fuse_main + fuse_fill"
    kd = kernels[dom]
    traffic = profiled_traffic() if trk.front_fused else None
    roofline = {"kernel": dom, "bound": "hbm", "achieved": round(kd["gbs"], 1), "peak": hbm, "unit": "GB/s",
                "frac": round(kd["gbs"] / hbm, 4), "traffic": traffic, "peak_source": hbm_src}
    value = job_value(K, ws, total_ms)
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": round(total_ms / K, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "tunnel 64x1024 sweeps vs 512x2048 FP32 keyframes, keyframe every 5 m, <=15 ICP iters",
                   "sweep": "64x1024", "keyframe": "512x2048 f32", "scans": K, "parallelism": f"replicas{ws}",
                   "l2": "flushed between steps (256 MiB write, outside the step events)",
                   "graph": used_graph},
        "roofline": roofline,
        "kernels": {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                    for k, v in kernels.items()},
        "gpu_launches": launches[0],
        "clocks": clocks,
        "accuracy": {"trans_err_m_median": float(np.median([e[0] for e in errs])),
                     "trans_err_m_max": float(np.max([e[0] for e in errs])),
                     "rot_err_deg_max": float(np.degrees(np.max([e[1] for e in errs]))),
                     "accepted": int(accepted), "icp_iters_avg": float(np.mean(iters))},
        "wall_s_timed": round(t_wall, 4),
    }
    if rank == 0 and args.e2e_steps > 0:
        out["e2e"] = run_e2e(args, seq, h_scans, device, up)
    if rank == 0 and args.atrous_levels > 0:
        k_fuse = min(kf_every - 1, n_scans - 1)  # a sweep registered against the first keyframe
        out["extra_kernels"] = {"atrous_kernel": run_atrous(args, seq, d_scans, device, up, hbm, hbm_src),
                                "grid_score_kernel": run_grid(trk, device, up, hbm, hbm_src),
                                "consistency_kernels": (run_consistency(pool, hist_pose[kf_every].clone(), device, up,
                                                                        hbm, hbm_src) if n_scans > kf_every else
                                                        run_consistency(switch_pair(trk, seq, device, up),
                                                                        trk.state.pose.clone(), device, up, hbm,
                                                                        hbm_src)),
                                "fuse_kernels": run_fuse(pool[0], seq, d_scans[k_fuse], hist_pose[k_fuse].clone(),
                                                         device, up, hbm, hbm_src),
                                "keyframe_switch": run_switch(trk, seq, device, up, hbm, hbm_src)}
    if dist:
        dist.barrier()
    return out


def _time_graph_diff(fn, reps, pre, warm=2):
    """Device ms of one fn() call by difference: a graph of reps x [pre(), fn()] and one of reps x [pre()],
    each replay timed between one pair of CUDA events, (T1 - T0) / reps (medians of 5 replays).  The calls
    run back to back as inside a stream of work, so the few microseconds an event pair adds around one
    short launch (about 6 us for an empty kernel on GB300) do not enter; pre() restores the inputs and
    flushes L2 before every call.  fn and pre must launch on torch's current stream."""
    import torch
    for _ in range(warm):
        pre()
        fn()
    torch.cuda.synchronize()

    def capture(with_fn):
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                for _ in range(reps):
                    pre()
                    if with_fn:
                        fn()
        torch.cuda.current_stream().wait_stream(s)
        return g

    def replay_ms(g):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        b.synchronize()
        return a.elapsed_time(b)

    g1, g0 = capture(True), capture(False)
    replay_ms(g1)
    replay_ms(g0)
    t1 = statistics.median(replay_ms(g1) for _ in range(5))
    t0 = statistics.median(replay_ms(g0) for _ in range(5))
    return (t1 - t0) / reps


def run_grid(trk, device, up, hbm, hbm_src):
    """Loop-closure grid search (Sec. III-C) on the tracker's last keyframe and sweep: 729 candidates
    (9 x 9 translations of 0.1 m x 9 yaws of 2 deg) around the last pose, keyframe sampled every 4 pixels.
    Work unit: a (sampled keyframe pixel, candidate) pair; its gather is 32 B of L2-resident sweep data."""
    import torch
    xi = []
    for i in range(9):
        for j in range(9):
            for k in range(9):
                xi.append([0.0, 0.0, math.radians((k - 4) * 2.0), (i - 4) * 0.1, (j - 4) * 0.1, 0.0])
    xi = torch.tensor(xi, dtype=torch.float32, device=device)
    poses = up.grid_candidates(trk.state.pose.clone(), xi)
    p = up.Params(d_max=0.1)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    ms = _time_graph_diff(lambda: up.grid_score(trk.kf, trk.sw, poses, p, 4), 20, flush.zero_)
    samples = int((trk.kf.depth[::4, ::4] > 0).sum().item())
    pairs = samples * poses.shape[0]
    # ALU roofline: the FP32 arithmetic a binned pair needs by its definition (an FMA counted once): the
    # inverse transform (12); the binning rule (59: the two ranges' squares, sums and square roots 7, two
    # atan2 polynomials of 23 each (the max / min, one division, the square, eight multiply-add pairs, the
    # product and two quadrant fixes), the column and row scalings 4 and their two floors); then the sweep
    # point and normal transformed and the two gate tests (27).  Against the SMs' FP32 issue rate, 128
    # lanes per SM per cycle at the 2070 MHz maximum SM clock
    ops_per_pair = 12 + 59 + 27
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    peak_tops = sms * 128 * 2.07e9 / 1e12
    tops = pairs * ops_per_pair / (ms * 1e-3) / 1e12
    return {"candidates": int(poses.shape[0]), "stride": 4, "sampled_keyframe_samples": samples,
            "launches": 2, "ms_avg": round(ms, 5), "pairs_per_s": round(pairs / (ms * 1e-3), 1),
            "bound": "alu (FP32 binning rule per pair) + L2 gathers", "l2": "flushed before each call",
            "roofline": {"bound": "alu", "achieved": round(tops, 2), "peak": round(peak_tops, 2),
                         "unit": "T FP32 ops/s", "frac": round(tops / peak_tops, 4),
                         "ops_per_pair": ops_per_pair,
                         "peak_source": f"{sms} SMs x 128 FP32 lanes x 2070 MHz (derived)"},
            "timing": DIFF_TIMING}


def switch_pair(trk, seq, device, up):
    """The two keyframes of a switch at the tracker's last sweep, as copies (the check removes samples): a copy
    of the current keyframe, and a new one hole-filled from the last sweep in that sweep's frame."""
    a = up.KeyframeBuffer(seq.kf, device)
    a.set(trk.kf.depth, trk.kf.nw)
    b = up.KeyframeBuffer(seq.kf, device)
    up.fuse(b, trk.sw, trk.identity, up.Params(accept_quality=0.1))
    return [a, b]


def run_consistency(pool, T_ab, device, up, hbm, hbm_src):
    """Keyframe mutual consistency check (Sec. III-C) between the first two 512 x 2048 keyframes of the run
    (T_ab: the registered pose of the sweep that started the second one, in the first), or, when the run
    opened no second keyframe, between the current one and one started from its last sweep.
    Algorithmic bytes per keyframe pixel and side: depth read (4 B), flag written (1 B) and read back (1 B);
    the neighbourhood gathers of the other keyframe hit L1/L2."""
    import ctypes
    import torch
    a, b = pool[0], pool[1]
    L = up.lib()
    ka, kb = a.struct(), b.struct()
    nbytes = int(L.upslam_consistency_workspace_bytes(ctypes.byref(ka), ctypes.byref(kb)))
    ws = torch.zeros(nbytes, dtype=torch.uint8, device=device)
    removed = torch.zeros(2, dtype=torch.int64, device=device)
    T = T_ab
    # repeated calls only remove what the first one did not: the timing is of the flag pass and a no-op apply
    args = (ctypes.byref(ka), ctypes.byref(kb), ctypes.c_void_p(T.data_ptr()), ctypes.c_float(0.05),
            ctypes.c_float(0.2), ctypes.c_void_p(ws.data_ptr()), ctypes.c_size_t(nbytes),
            ctypes.c_void_p(removed.data_ptr()))
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def fn():
        rc = L.upslam_keyframe_consistency(*args, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, rc

    ms = _time_graph_diff(fn, 20, flush.zero_)
    px = int(a.depth.numel() + b.depth.numel())
    nbytes_alg = px * 6
    gbs = nbytes_alg / (ms * 1e-3) / 1e9
    return {"pixels": px, "launches": 2, "ms_avg": round(ms, 5), "bytes": nbytes_alg, "gbs": round(gbs, 1),
            "bound": "hbm", "peak": hbm, "frac": round(gbs / hbm, 4), "peak_source": hbm_src,
            "timing": DIFF_TIMING, "l2": "flushed before each call"}


def run_switch(trk, seq, device, up, hbm, hbm_src, reps=20):
    """A keyframe switch (Sec. III-C, a new keyframe every 5 m) timed alone through the public API:
    ``Tracker.new_keyframe(buffer=..., consistency=True)`` on the tracker's last sweep, i.e. the
    sweep's hole fill into an empty 512 x 2048 keyframe (two launches) and the mutual consistency
    check between the keyframe being left and the new one (workspace clear and two launches).  The
    keyframe being left is restored and the new one cleared before each call, and L2 is flushed,
    all outside the events."""
    import torch
    old = trk.kf
    d0, n0 = old.depth.clone(), old.nw.clone()
    prev0 = trk.prev.clone()
    new = up.KeyframeBuffer(seq.kf, device)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def pre():
        trk.kf = old
        old.set(d0, n0)
        new.clear()
        flush.zero_()

    removed = []

    def fn():
        trk.new_keyframe(buffer=new, consistency=True)
        removed.append(trk.last_removed)

    ms = _time_graph_diff(fn, reps, pre)
    trk.kf = old
    old.set(d0, n0)
    trk.prev.copy_(prev0)
    px = int(old.depth.numel())
    # hole fill: sweep read (32 B/px) + every new keyframe pixel written once (20 B); consistency: both
    # keyframes' depth read (4 B/px) and flags written and read (2 B/px)
    alg = seq.sweep.pixels * 32 + px * 20 + 2 * px * 6
    gbs = alg / (ms * 1e-3) / 1e9
    rem = removed[-1].cpu().tolist() if removed else None
    return {"ms_avg": round(ms, 5), "launches": 4, "bytes": alg, "gbs": round(gbs, 1), "bound": "hbm", "peak": hbm,
            "frac": round(gbs / hbm, 4), "peak_source": hbm_src, "samples_removed": rem,
            "timing": DIFF_TIMING, "l2": "flushed before each call",
            "note": "one switch per 50 sweeps in the headline sequence"}


def run_fuse(kf, seq, scan, T, device, up, hbm, hbm_src, reps=20):
    """Keyframe update (Sec. III-C) timed alone through the C ABI (`upslam_fuse`: the averaging + hole-fill
    atomics launch, then the hole-fill write launch): one sweep fused into a 512 x 2048 FP32 keyframe of
    the run at its registered pose T.  Before every call the keyframe is put back to its saved state and
    L2 is flushed, both outside the events, so each call does the same work from DRAM.
    Algorithmic bytes per call: every keyframe pixel read once (depth 4 B + normal and count 16 B), every
    pixel the call changes written once (20 B), each sweep pixel's point and normal read by both launches
    (2 x 32 B)."""
    import torch
    p = up.Params(accept_quality=0.1)
    sw = up.SweepFrame(seq.sweep, device)
    sw.load(scan, p)
    d0, n0 = kf.depth.clone(), kf.nw.clone()
    up.fuse(kf, sw, T, p)
    changed = int(((kf.depth != d0) | (kf.nw != n0).any(-1)).sum())
    samples = int((n0[..., 3] > 0).sum())
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def pre():
        kf.depth.copy_(d0)
        kf.nw.copy_(n0)
        flush.zero_()

    ms = _time_graph_diff(lambda: up.fuse(kf, sw, T, p), reps, pre)
    kf.depth.copy_(d0)
    kf.nw.copy_(n0)
    kf_px, sw_px = kf.depth.numel(), seq.sweep.pixels
    # the algorithmic bytes: every keyframe pixel read and written once (20 B each way) and the
    # hole fill's read of the sweep (24 B per sweep pixel)
    nbytes = kf_px * 40 + sw_px * 24
    touched = kf_px * 20 + changed * 20 + sw_px * 64
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"keyframe": f"{int(seq.kf.rows)}x{int(seq.kf.cols)} f32", "samples_before": samples,
            "pixels_written": changed, "launches": 2, "ms_avg": round(ms, 5), "bytes": nbytes,
            "gbs": round(gbs, 1), "bound": "hbm", "peak": hbm, "frac": round(gbs / hbm, 4),
            "peak_source": hbm_src, "bytes_touched": touched,
            "timing": DIFF_TIMING,
            "l2": "flushed before each call (keyframe restored first)"}


def run_atrous(args, seq, d_scans, device, up, hbm, hbm_src):
    """The a-trous normal smoothing (Sec. III-A) on the workload's sweeps, timed alone through the C ABI.

    Each repetition loads a different sweep (project + normals, untimed), flushes L2, then times the
    smoothing launches with CUDA events on the launching stream.  Algorithmic bytes per level and
    pixel: the normal read (16 B), the point read (16 B) and the normal written (16 B)."""
    import ctypes
    import torch
    levels = args.atrous_levels
    p = up.Params(accept_quality=0.1, atrous_levels=levels)
    sw = up.SweepFrame(seq.sweep, device)
    raw = torch.zeros_like(sw.nrm)
    out = torch.zeros_like(sw.nrm)
    tmp = torch.zeros_like(sw.nrm)
    ps = up.pano_struct(seq.sweep)
    ap = p.atrous()
    L = up.lib()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    reps = min(50, d_scans.shape[0])
    rep = [0]

    def pre():
        sw.load(d_scans[rep[0] % d_scans.shape[0]], up.Params(accept_quality=0.1))
        rep[0] += 1
        raw.copy_(sw.nrm)
        flush.zero_()

    def fn():
        st = torch.cuda.current_stream().cuda_stream
        rc = L.upslam_atrous_normals(ctypes.byref(ps), ctypes.c_void_p(sw.pix.data_ptr()),
                                     ctypes.c_void_p(raw.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(tmp.data_ptr()), up.F32, ctypes.byref(ap), ctypes.c_void_p(st))
        assert rc == 0, rc

    ms = _time_graph_diff(fn, reps, pre)
    px = seq.sweep.pixels
    bytes_level = px * 48
    gbs = bytes_level * levels / (ms * 1e-3) / 1e9
    return {"levels": levels, "launches": levels, "ms_avg": round(ms, 5), "us_per_level": round(ms * 1e3 / levels, 3),
            "bytes_per_level": bytes_level, "gbs": round(gbs, 1), "bound": "hbm", "peak": hbm,
            "frac": round(gbs / hbm, 4), "peak_source": hbm_src, "reps": reps,
            "timing": DIFF_TIMING, "l2": "flushed before each repetition (outside the timed calls)"}


def run_e2e(args, seq, h_scans, device, up):
    """Public API from pinned host memory, driven as a streaming caller would: every step copies its sweep
    host -> device (on a copy stream, overlapping the previous sweep's tracking), tracks it, copies its pose and
    record device -> host, and the host reads that result while the next sweep runs.  All copies of every step
    are inside the timed region."""
    import torch
    K = min(args.e2e_steps, h_scans.shape[0] - 1)
    p = up.Params(accept_quality=0.1)
    trk = up.Tracker(seq.sweep, seq.kf, p, device=device, constant_velocity=True)
    n_kf = 2 + K // seq.kf_every
    pool = [trk.kf] + [up.KeyframeBuffer(seq.kf, device) for _ in range(n_kf)]
    staging = [torch.empty(h_scans.shape[1:], dtype=torch.float32, device=device) for _ in range(2)]
    out_pose = [torch.empty(12, dtype=torch.float64).pin_memory() for _ in range(2)]
    out_stats = [torch.empty(up._abi.STATS_BYTES, dtype=torch.uint8).pin_memory() for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]  # sweep copied into staging[b]
    free = [torch.cuda.Event() for _ in range(2)]   # the sweep in staging[b] has been tracked
    done = [torch.cuda.Event() for _ in range(2)]   # pose and record of the step in out_*[b]
    cs = torch.cuda.Stream(device=device)
    ms = torch.cuda.current_stream()
    staging[0].copy_(h_scans[0], non_blocking=True)
    trk.new_keyframe(staging[0])
    torch.cuda.synchronize()

    def h2d(k):
        b = k % 2
        with torch.cuda.stream(cs):
            if k >= 3:
                cs.wait_event(free[b])
            staging[b].copy_(h_scans[k], non_blocking=True)
            ready[b].record(cs)

    pos = 0
    checksum = 0.0
    t0 = time.perf_counter()
    h2d(1)
    for k in range(1, K + 1):
        b = k % 2
        if k < K:
            h2d(k + 1)
        ms.wait_event(ready[b])
        trk.track(staging[b])
        free[b].record(ms)
        if k % seq.kf_every == 0:
            pos += 1
            trk.new_keyframe(buffer=pool[pos])
        out_pose[b].copy_(trk.state.pose, non_blocking=True)
        out_stats[b].copy_(trk.state.stats, non_blocking=True)
        done[b].record(ms)
        if k >= 2:  # the previous step's result, read while this step runs
            done[1 - b].synchronize()
            checksum += float(out_pose[1 - b][3])
    done[K % 2].synchronize()
    checksum += float(out_pose[K % 2][3])
    dt = time.perf_counter() - t0
    return {"value": round(K / dt, 2), "unit": UNIT, "steps": K,
            "h2d_bytes_per_step": int(h_scans[0].numel() * 4),
            "d2h_bytes_per_step": int(12 * 8 + up._abi.STATS_BYTES),
            "overlap": "sweep k+1 copied in on a second stream while sweep k tracks; step k's result read on "
                       "the host while step k+1 runs",
            "l2": "not flushed between steps: the keyframe stays cache-resident across sweeps, as for a "
                  "streaming caller (the device-timed value flushes L2 before every step)"}


# ----------------------------------------------------------------------------- oracle timing

def oracle_rate(seq, scans, budget_s: float, warm: int = 1, max_steps: int | None = None):
    """Sweeps/s of the FP64 oracle over consecutive sweeps, within a time budget."""
    import oracle
    import synth
    prm = oracle.Params(accept_quality=0.1)
    I = np.hstack([np.eye(3), np.zeros((3, 1))])
    kf = oracle.Keyframe(seq.kf)
    sp, sn, _, _ = oracle.sweep_frame(scans[0], seq.sweep, prm)
    oracle.fuse(kf, sp, sn, seq.sweep, I, prm)
    T_prev, M = I.copy(), I.copy()

    def one(k):
        nonlocal kf, T_prev, M
        T0 = synth.pose_mul(T_prev, M)
        u, _, vt = np.linalg.svd(T0[:, :3])
        T0[:, :3] = u @ vt
        T, st, it, acc = oracle.process_scan(kf, scans[k], seq.sweep, T0, prm)
        M = synth.pose_mul(synth.pose_inv(T_prev), T)
        T_prev = T
        if k % seq.kf_every == 0:
            kf = oracle.Keyframe(seq.kf)
            sp, sn, _, _ = oracle.sweep_frame(scans[k], seq.sweep, prm)
            oracle.fuse(kf, sp, sn, seq.sweep, I, prm)
            T_prev = I.copy()

    k = 1
    for _ in range(warm):
        one(k)
        k += 1
    n = 0
    t0 = time.perf_counter()
    while k < len(scans) and (max_steps is None or n < max_steps):
        one(k)
        k += 1
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    W = max(1, args.warmup)
    n = 1 + W + min(args.steps, 400)
    seq, scans = make_workload(n, rank)
    rate, steps, dt = oracle_rate(seq, scans, budget_s=150.0, warm=W, max_steps=args.steps)
    sample = (f"the first {steps} sweeps after {W} warm-up sweeps of the tunnel sequence (whole path per sweep), "
              f"capped at 150 s of CPU time")
    return {"impl": "reference", "metric": METRIC, "value": round(rate, 4), "unit": UNIT, "n_gpus": ws,
            "steps": steps, "warmup": W, "ms_per_step": round(dt / max(steps, 1) * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "tunnel 64x1024 sweeps vs 512x2048 FP32 keyframes, keyframe every 5 m, <=15 ICP "
                                   "iters", "parallelism": "single host thread"},
            "cpu_baseline": {"value": round(rate, 4), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(rate, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_campus(args, local):
    """Precision form: 128x2048 campus sweeps vs 1024x4096 keyframes, FP16 normals and counts."""
    import torch
    import paper_2101_00585_gb300 as up
    from synth import configs
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    W, K = args.warmup, min(args.steps, args.form_steps)
    seq = configs.campus_sequence(n_scans=1 + W + K)
    scans = np.stack([seq.scan(k) for k in range(1 + W + K)])
    d_scans = torch.from_numpy(scans).to(device)
    trk = up.Tracker(seq.sweep, seq.kf, up.Params(accept_quality=0.1), precision=up.F16, device=device)
    pool = [trk.kf] + [up.KeyframeBuffer(seq.kf, device, up.F16) for _ in range(2 + (1 + W + K) // seq.kf_every)]
    pos = [0]
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def step(k):
        trk.track(d_scans[k])
        if k % seq.kf_every == 0:
            pos[0] += 1
            trk.new_keyframe(buffer=pool[pos[0]])

    trk.new_keyframe(d_scans[0])
    for k in range(1, 1 + W):
        step(k)
    torch.cuda.synchronize()
    # the timed sweeps as one captured graph, as the headline: an event node pair around each sweep's
    # launches, the L2 flush between sweeps outside them; the records are copied out per sweep
    cr = Cudart()
    cr.external = True
    evs = [(cr.event(), cr.event()) for _ in range(K)]
    hist = torch.zeros((K, up._abi.STATS_BYTES), dtype=torch.uint8, device=device)
    s = torch.cuda.Stream(device)
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    saved = pos[0]
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            st = torch.cuda.current_stream().cuda_stream
            for i in range(K):
                flush.zero_()
                cr.record(evs[i][0], st)
                step(1 + W + i)
                cr.record(evs[i][1], st)
                hist[i].copy_(trk.state.stats)
        pos[0] = saved
        g.replay()
    torch.cuda.synchronize()
    ms = [cr.elapsed(a, b) for a, b in evs]
    total = float(sum(ms))
    from paper_2101_00585_gb300._abi import IcpStats
    raw = hist.cpu().numpy()
    iters = [IcpStats.from_buffer_copy(bytes(raw[i])).iters for i in range(K)]
    kf_px, sw_px = seq.kf.pixels, seq.sweep.pixels
    # the algorithmic bytes: the FP16 keyframe read and written once (12 B each way per pixel) and, per
    # Gauss-Newton step, the sweep pixel's point, normal and the keyframe sample (16 + 8 + 12 B per sweep pixel)
    bytes_track = kf_px * 24 + sw_px * 36 * float(np.mean(iters))
    hbm, src = peaks()
    gbs = bytes_track * K / (total * 1e-3) / 1e9
    return {"metric": "ICP+fusion scans/s at 128x2048 vs 1024x4096 FP16 keyframes (precision form)",
            "value": round(K / (total * 1e-3), 2), "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W,
            "ms_per_step": round(total / K, 4), "higher_is_better": True, "dtype": "f32 arithmetic, f16 normals/counts",
            "data": "synthetic", "config": {"workload": "campus 128x2048 sweeps vs 1024x4096 keyframes, FP16 storage",
                                            "l2": "flushed between steps", "graph": True},
            "roofline_step": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                              "frac": round(gbs / hbm, 4), "peak_source": src,
                              "bytes_per_step": round(bytes_track)},
            "icp_iters_avg": float(np.mean(iters))}


def run_forest_batch(args, local):
    """Batched form: one 64x1024 forest sweep vs 64 keyframes (22 x 256x1024, 21 x 512x2048,
    21 x 1024x4096) x 8 hypotheses up to 2 m / 20 deg = 512 problems in one persistent launch,
    captured once as a CUDA graph and replayed.  The Omega gate is coarse-to-fine: 1.0 m for five
    Gauss-Newton steps, then 0.5 m.

    Algorithmic bytes per launch: every keyframe pixel read once by the staging prologue (depth 4 B +
    normal and count 16 B), then per problem and step the sweep pixel each of the keyframe's samples
    bins into (point 16 B + normal 16 B).  The same bytes by a coarser per-iteration estimate
    (0.67 GB per step over all 64 keyframes) are reported beside it."""
    import torch
    import paper_2101_00585_gb300 as up
    from paper_2101_00585_gb300 import autotune
    import synth
    from synth import configs
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    n_kf = args.batch_keyframes
    case = configs.forest_batch() if n_kf == 64 else configs.forest_batch(
        n_kf=n_kf, kf_sizes=tuple(((256, 1024), (512, 2048), (1024, 4096))[i % 3] for i in range(n_kf)))
    p = up.Params(max_iters=15, d_max=1.0, coarse_iters=5, d_max_fine=0.5)
    sw = up.SweepFrame(case.sweep, device)
    sw.load(torch.from_numpy(case.scan).to(device), p)
    bufs = []
    builder = up.SweepFrame(case.sweep, device)
    I = up.identity_pose(device)
    for i, (P_kf, kp) in enumerate(zip(case.kf_poses, case.kf_panos)):
        sc = synth.scan(case.scene, case.lidar, P_kf, np.random.default_rng((4, 100 + i)))
        builder.load(torch.from_numpy(sc).to(device), p)
        b = up.KeyframeBuffer(kp, device)
        up.fuse(b, builder, I, p, None)
        bufs.append(b)
    batch = up.Batch(sw, bufs, case.n_hyp)
    init = torch.from_numpy(np.stack([np.asarray(h).reshape(12) for hyps in case.T_init for h in hyps])).to(device)
    tuned = ({"tiles": [512, 512], "ms": {}} if args.no_autotune else autotune.tune(batch, init, p, reps=2))
    batch.run(init, p)  # first launch outside the capture
    batch.capture(p)
    batch.init.copy_(init)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    for _ in range(max(1, args.warmup)):
        batch.replay()
    torch.cuda.synchronize()
    K = max(1, min(args.steps, 50))
    ms = []
    for _ in range(K):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        batch.replay()
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    recs = batch.read_stats()
    poses = batch.poses.cpu().numpy().reshape(-1, 3, 4)
    ok = 0
    for q in range(batch.n_prob):
        k = q // case.n_hyp
        dt, dr = synth.pose_error(poses[q], case.T_true[k])
        ok += dt < 0.02 and dr < math.radians(0.1)
    avg = statistics.mean(ms)
    samples = [int((b.nw[..., 3] > 0).sum()) for b in bufs]
    kf_bytes = sum(int(b.depth.numel()) for b in bufs) * 20
    steps_by_problem = [r["iters"] for r in recs]
    gather_bytes = sum(steps_by_problem[q] * samples[q // case.n_hyp] * 32 for q in range(batch.n_prob))
    alg = kf_bytes + gather_bytes
    est_bytes = 0.67e9 * float(np.mean(steps_by_problem))
    hbm, src = peaks()
    gbs = alg / (avg * 1e-3) / 1e9
    return {"metric": "batched ICP problems/s (64 keyframes x 8 hypotheses, one launch)",
            "value": round(batch.n_prob / (avg * 1e-3), 1), "unit": "problems/s", "n_gpus": 1, "steps": K,
            "ms_per_launch": round(avg, 3), "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "graph": True, "gpu_launches_per_replay": 2,
            "config": {"workload": (f"forest: 64 keyframes (22x256x1024, 21x512x2048, 21x1024x4096) x 8 hypotheses "
                                    f"up to 2 m / 20 deg, keyframes started from a sweep each" if n_kf == 64 else
                                    f"forest: {n_kf} keyframes (256x1024, 512x2048, 1024x4096 in turn) x 8 "
                                    f"hypotheses up to 2 m / 20 deg"),
                       "gate": "d_max 1.0 m for 5 steps, then 0.5 m", "tiles": tuned["tiles"],
                       "autotune_ms": tuned["ms"], "l2": "flushed between launches"},
            "roofline": {"kernel": "icp_batched_kernel", "bound": "hbm", "achieved": round(gbs, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(gbs / hbm, 4), "bytes_per_launch": alg,
                         "peak_source": src,
                         "per_iteration_estimate": {"bytes_per_launch": round(est_bytes),
                                                    "frac": round(est_bytes / (avg * 1e-3) / 1e9 / hbm, 4)}},
            "samples_per_keyframe_mean": float(np.mean(samples)),
            "iters_avg": float(np.mean(steps_by_problem)),
            "within_2cm_0.1deg": int(ok), "problems": batch.n_prob}


def run_room(args, local):
    """Workload 1, a latency case: a 16 x 512 sweep of the box room (8192 points) registered against a
    256 x 512 keyframe rendered from a second pose 5 cm / 2 deg away, 10 Gauss-Newton steps, then fused.
    Reports microseconds per whole sweep (one upslam_track_scan launch: projection, normals, ICP,
    keyframe update; the keyframe is restored before each call) and per ICP step (upslam_icp with ten
    forced steps, divided by ten).  Not a roofline case: the work is too small to fill the GPU."""
    import torch
    import paper_2101_00585_gb300 as up
    import synth
    from synth import configs
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    c = configs.room_case(noise=True)
    p = up.Params(max_iters=10, accept_quality=0.1)
    d, _, _ = synth.render_keyframe(c.scene, c.kf, c.P_w_kf)
    depth = torch.from_numpy(d.astype(np.float32)).to(device)
    trk = up.Tracker(c.sweep, c.kf, p, device=device, constant_velocity=False)
    pix = up.unproject(depth, c.kf, trk.kf.dirs)
    nrm = up.normals(pix, depth, c.kf, p)
    nrm[..., 3] = (depth > 0).float()
    trk.kf.set(depth, nrm)
    d0, n0 = trk.kf.depth.clone(), trk.kf.nw.clone()
    scan = torch.from_numpy(c.scan).to(device)
    K = max(10, min(args.steps, 200))
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    cr = Cudart()
    cr.external = False
    st = torch.cuda.current_stream().cuda_stream

    def pre():
        trk.kf.set(d0, n0)
        trk.prev.copy_(trk.identity)
        flush.zero_()

    scan_us = 1e3 * _time_graph_diff(lambda: trk.track(scan), 20, pre)
    evs = [(cr.event(), cr.event()) for _ in range(K)]
    iters = []
    for i in range(K + 3):
        pre()
        if i >= 3:
            cr.record(evs[i - 3][0], st)
        trk.track(scan)
        if i >= 3:
            cr.record(evs[i - 3][1], st)
            iters.append(trk.state.read_stats()["iters"])
    torch.cuda.synchronize()
    eager_us = 1e3 * statistics.median(cr.elapsed(a, b) for a, b in evs)
    err = synth.pose_error(trk.state.pose.cpu().numpy().reshape(3, 4), c.T_true)
    # ICP steps alone: the same sweep, ten forced steps per launch
    trk.kf.set(d0, n0)
    trk.sw.load(scan, p)
    state = up.IcpState(trk.kf, device)
    p10 = up.Params(max_iters=10, eps_rot=0.0, eps_trans=0.0)
    def pre_icp():
        state.pose.copy_(trk.identity)
        flush.zero_()

    icp_us = 1e3 * _time_graph_diff(lambda: up.icp(trk.kf, trk.sw, state, p10), 20, pre_icp)
    cpu = None
    if not args.no_cpu_baseline:
        # the FP64 oracle on the same registration: sweep frame, 10 Gauss-Newton steps, keyframe update
        import oracle
        prm = oracle.Params(max_iters=10, accept_quality=0.1)
        kd = d.astype(np.float32)
        kn, kv = oracle.normals(oracle.keyframe_points(kd, c.kf).astype(np.float32), kd, c.kf, prm)
        kn4 = oracle.normals4(kn, kv)
        reps, t0 = 3, time.perf_counter()
        for _ in range(reps):
            kf_ref = oracle.Keyframe(c.kf, kd.astype(np.float64), kn4[..., :3].astype(np.float64),
                                     (kd > 0).astype(np.float64))
            oracle.process_scan(kf_ref, c.scan, c.sweep, np.hstack([np.eye(3), np.zeros((3, 1))]), prm)
        dt = (time.perf_counter() - t0) / reps
        cpu = {"value": round(dt * 1e6, 1), "unit": "us per sweep", "cores": 1, "kind": "oracle",
               "sample": f"the same room registration, {reps} repetitions on one host thread"}
    return {"metric": "latency of one 16x512 room sweep vs a 256x512 keyframe", "unit": "us",
            "higher_is_better": False, "us_per_scan": round(scan_us, 2), "us_per_icp_step": round(icp_us / 10, 3),
            "us_per_scan_eager": round(eager_us, 2),
            "icp_launch_us_10_steps": round(icp_us, 2), "icp_iters_avg": float(np.mean(iters)), "reps": K,
            "pose_error_m": float(err[0]), "pose_error_deg": float(math.degrees(err[1])), "cpu_baseline": cpu,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "room 16x512 sweep (8192 points) vs 256x512 keyframe, 5 cm / 2 deg, <=10 steps",
                       "l2": "flushed before each call",
                       "timing": "device time by difference of graph replays (" + DIFF_TIMING + "); us_per_scan_eager: "
                                 "one eager call between two events on an idle stream, median of reps"}}


def run_learned(args, local):
    """Learned-proposal form: train on pairs the plain pipeline makes, then learned + ICP vs plain + ICP."""
    import torch
    import paper_2101_00585_gb300 as up  # noqa: F401
    from paper_2101_00585_gb300 import proposal
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    x, xi, _ = proposal.make_pairs(args.train_pairs, seed=20210106)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    net = proposal.PoseNet(256)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    hist = proposal.train(net, x, xi, epochs=args.epochs, lr=2e-3, seed=7, log=log)
    b.record()
    b.synchronize()
    t_train = a.elapsed_time(b) * 1e-3
    steps = args.epochs * (args.train_pairs // net.batch)
    pairs_trained = steps * net.batch
    flops = pairs_trained * 0.34e9  # forward 0.113 GFLOP + backward about twice that, per pair
    step_bytes = cnn_step_bytes(net.batch)
    del x
    xt, xit, ext = proposal.make_pairs(args.eval_pairs, seed=20210107, keep_scans=True)
    # the learned start is close, so its ICP gets fewer Gauss-Newton steps (12 of the plain start's 15); the
    # same evaluation with 15 steps from the learned start is reported beside it
    res = proposal.evaluate(net, xt, ext["motions"], ext["scans"], learned_max_iters=LEARNED_ICP_STEPS)
    full = proposal.evaluate(net, xt, ext["motions"], ext["scans"])
    peak, peak_src = bf16_peak("sustained")  # training is a seconds-long loop of GEMMs
    hbm_peak, hbm_src = peaks()
    return {"metric": "learned-init vs plain-init ICP success within 2 cm / 0.1 deg (held-out pairs)",
            "value": res["gated_success"] / res["pairs"], "unit": "fraction of pairs", "higher_is_better": True,
            "plain_fraction": res["plain_success"] / res["pairs"], "learned_only_fraction":
                res["learned_success"] / res["pairs"], "fallbacks": res["fallbacks"], "pairs": res["pairs"],
            "plain_pairs_per_s": round(res["plain_pairs_per_s"], 1),
            "gated_pairs_per_s": round(res["gated_pairs_per_s"], 1),
            "pairs_per_s_basis": "device time of the ICP launches (+ the network forward for the gated path)",
            "plain_pairs_per_s_wall": round(res["plain_pairs_per_s_wall"], 1),
            "gated_pairs_per_s_wall": round(res["gated_pairs_per_s_wall"], 1),
            "icp_steps_per_pair_plain": round(res["icp_steps_per_pair_plain"], 2),
            "icp_steps_per_pair_gated": round(res["icp_steps_per_pair_gated"], 2),
            "cnn_ms_per_pair": res["cnn_ms_per_pair"], "learned_icp_steps_max": LEARNED_ICP_STEPS,
            "learned_15_steps": {"fraction": full["gated_success"] / full["pairs"],
                                 "gated_pairs_per_s": round(full["gated_pairs_per_s"], 1),
                                 "fallbacks": full["fallbacks"]},
            "train": {"pairs": args.train_pairs, "epochs": args.epochs, "batch": net.batch, "loss": hist,
                      "seconds": round(t_train, 2), "ms_per_step": round(t_train * 1e3 / max(1, steps), 3),
                      "pairs_per_s": round(pairs_trained / t_train, 1),
                      "tflops": round(flops / t_train / 1e12, 2),
                      "frac_of_bf16_peak": round(flops / t_train / 1e12 / peak, 5),
                      "bf16_peak_tflops": peak, "peak_source": peak_src,
                      "hbm": {"bytes_per_step": step_bytes,
                              "achieved_gbs": round(step_bytes * steps / t_train / 1e9, 1),
                              "frac": round(step_bytes * steps / t_train / 1e9 / hbm_peak, 4), "peak": hbm_peak,
                              "peak_source": hbm_src,
                              "basis": "each BF16 activation and gradient tensor read or written once per use "
                                       "(mini-batch gather, forward, backward); weights not counted"},
                      "pair_generation_s": round(t_gen, 1)},
            "dtype": "bf16 weights/activations, f32 accumulate", "data": "synthetic",
            "config": {"workload": "tunnel/forest/road pairs, motion <= 1 m / 30 deg, 64x256 inputs"}}


def cnn_step_bytes(batch):
    """Compulsory DRAM bytes of one pose-network training step: every BF16 activation and gradient tensor
    read or written once per use.  Inputs [B, 64, 256, 8]; layer l writes [B, 64 >> (l+1), 256 >> (l+1), C].
    Forward: read the input, write each layer's output, read it as the next layer's input (the last by the
    pool).  Backward: write the last dY; per layer the weight gradient reads its input and dY, and the data
    gradient (layers 2-4) reads dY and the ReLU mask and writes the dY below.  Plus the mini-batch gather
    (the inputs read from the pool and written to the batch)."""
    chans = [8, 32, 64, 128, 128]
    x0 = batch * 64 * 256 * 8 * 2
    act = [batch * (64 >> (l + 1)) * (256 >> (l + 1)) * chans[l + 1] * 2 for l in range(4)]
    fwd = x0 + sum(act) + sum(act)
    bwd = act[3]
    for l in range(3, -1, -1):
        bwd += (x0 if l == 0 else act[l - 1]) + act[l]
        if l > 0:
            bwd += act[l] + act[l - 1] + act[l - 1]
    return fwd + bwd + 2 * x0


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "ours" and args.workload != "tunnel":
        runner = {"room": run_room, "campus": run_campus, "forest-batch": run_forest_batch,
                  "learned": run_learned}[args.workload]
        out = runner(args, local)
        print(json.dumps(out), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out = run_ours(args, ws, rank, local)
    if rank == 0 and not args.no_cpu_baseline:
        seq, scans = make_workload(1 + 40, rank)
        rate, n, dt = oracle_rate(seq, scans, budget_s=args.cpu_seconds, warm=1)
        out["cpu_baseline"] = {"value": round(rate, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"{n} consecutive tunnel sweeps (whole path each) after 1 warm-up, "
                                         f"{dt:.1f} s on one host thread"}
    if rank == 0 and args.forms == "all":
        out["forms"] = run_forms(args, local)
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_forms(args, local) -> dict:
    """The other workloads, each timed on its own after the headline (rank 0 only)."""
    forms = {}
    for name, fn in (("room", run_room), ("campus", run_campus), ("forest_batch", run_forest_batch),
                     ("learned", run_learned)):
        t0 = time.perf_counter()
        try:
            forms[name] = fn(args, local)
        except Exception as e:  # one form failing must not lose the headline line
            forms[name] = {"error": f"{type(e).__name__}: {e}"}
        forms[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        log(f"[bench] form {name}: {forms[name].get('value', forms[name].get('us_per_scan'))}")
    return forms


if __name__ == "__main__":
    main()
