"""Batched persistent form (workload 4): one forest sweep against keyframes of mixed sizes, several
initial-pose hypotheses per keyframe, all problems in one cooperative launch.

Keyframes are started from a sweep taken at the keyframe's pose (the oracle's hole fill).  The batched launch
must agree with the oracle:
* one Gauss-Newton step for every problem: J^T J relative 1e-5, pose 1e-4 m / 1e-5 rad;
* a full registration on the small keyframes.

It must also agree with the single-problem launch (`upslam_icp`) on every problem, and the autotuner must pick
one of its candidates.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
import synth
from synth import configs
from tests.helpers import IDENTITY

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
up = pytest.importorskip("paper_2101_00585_gb300")

SIZES = ((256, 1024), (512, 2048), (1024, 4096), (256, 1024), (512, 2048), (1024, 4096))


def _upper(a):
    A = np.zeros((6, 6))
    A[np.triu_indices(6)] = a
    return A + np.triu(A, 1).T


def _keyframe(case, i, prm):
    """Keyframe i started from a sweep taken at its pose (the oracle's hole fill)."""
    sc = synth.scan(case.scene, case.lidar, case.kf_poses[i], np.random.default_rng((4, 100 + i)))
    kp_sweep, kn_sweep, _, _ = oracle.sweep_frame(sc, case.sweep, prm)
    kf = oracle.Keyframe(case.kf_panos[i])
    oracle.fuse(kf, kp_sweep, kn_sweep, case.sweep, IDENTITY, prm)
    return kf


@pytest.fixture(scope="module")
def forest():
    case = configs.forest_batch(n_kf=len(SIZES), n_hyp=4, max_trans=0.3, max_rot_deg=3.0, kf_sizes=SIZES)
    prm = oracle.Params()
    sp, sn, _, _ = oracle.sweep_frame(case.scan, case.sweep, prm)
    kfs = [_keyframe(case, i, prm) for i in range(len(SIZES))]
    return case, prm, sp, sn, kfs


# the row's own workload: 64 keyframes (22 x 256x1024, 21 x 512x2048, 21 x 1024x4096) x 8 hypotheses up to
# 2 m / 20 deg, gated coarse-to-fine (1.0 m for 5 steps, then 0.5 m)
FULL = dict(d_max=1.0, coarse_iters=5, d_max_fine=0.5)


@pytest.fixture(scope="module")
def forest_full():
    case = configs.forest_batch()
    prm = oracle.Params(**FULL)
    sp, sn, _, _ = oracle.sweep_frame(case.scan, case.sweep, prm)
    # the oracle's C calls release the interpreter lock, so threads build the keyframes side by side
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        kfs = list(ex.map(lambda i: _keyframe(case, i, prm), range(len(case.kf_panos))))
    return case, prm, sp, sn, kfs


def _gpu_batch(case, sp, sn, kfs, n_hyp):
    sw = up.SweepFrame(case.sweep)
    sw.set(torch.from_numpy(sp).cuda(), torch.from_numpy(sn).cuda())
    bufs = []
    for kf in kfs:
        b = up.KeyframeBuffer(kf.pp)
        b.set(torch.from_numpy(kf.depth_f32()).cuda(), torch.from_numpy(kf.nrm4_f32()).cuda())
        bufs.append(b)
    return sw, bufs, up.Batch(sw, bufs, n_hyp)


def _init(case):
    return torch.from_numpy(np.stack([np.asarray(h).reshape(12) for hyps in case.T_init for h in hyps])).cuda()


def test_batched_one_step_matches_oracle(forest):
    case, prm, sp, sn, kfs = forest
    sw, bufs, batch = _gpu_batch(case, sp, sn, kfs, case.n_hyp)
    init = _init(case)
    batch.run(init, up.Params(max_iters=1))
    recs = batch.read_stats()
    poses = batch.poses.cpu().numpy().reshape(-1, 3, 4)
    for p in range(batch.n_prob):
        k, h = divmod(p, case.n_hyp)
        T0 = case.T_init[k][h]
        Tn, st = oracle.icp_step(kfs[k].depth_f32(), kfs[k].nrm4_f32(), kfs[k].pp, sp, sn, case.sweep, T0, prm)
        A, A_ref = _upper(recs[p]["A"]), _upper(st["A"])
        assert np.linalg.norm(A - A_ref) <= 1e-5 * np.linalg.norm(A_ref), p
        assert abs(recs[p]["inliers"] - st["inliers"]) <= 2
        assert recs[p]["valid"] == st["valid"]
        if st["status"] == 0:
            dt, dr = synth.pose_error(poses[p], Tn)
            assert dt < 1e-4 and dr < 1e-5, (p, dt, dr)
        else:
            assert recs[p]["status"] == st["status"]


def test_batched_full_registration_matches_single_and_oracle(forest):
    case, prm, sp, sn, kfs = forest
    sw, bufs, batch = _gpu_batch(case, sp, sn, kfs, case.n_hyp)
    init = _init(case)
    p15 = up.Params(max_iters=15)
    batch.run(init, p15)
    recs = batch.read_stats()
    poses = batch.poses.cpu().numpy().reshape(-1, 3, 4)
    mismatched = 0
    for p in range(batch.n_prob):
        k, h = divmod(p, case.n_hyp)
        single = up.IcpState(bufs[k])
        single.pose.copy_(init[p])
        up.icp(bufs[k], sw, single, p15)
        dt, dr = synth.pose_error(poses[p], single.pose.cpu().numpy().reshape(3, 4))
        if not (dt < 1e-4 and dr < 1e-5):
            mismatched += 1
        assert recs[p]["iters"] >= 1
    # the two launch forms sum in different orders; a near-tie flipping one association may move one problem
    assert mismatched <= 1
    # the small keyframes against the oracle's full iteration, and against the truth
    for k in (0, 3):
        for h in range(case.n_hyp):
            p = k * case.n_hyp + h
            T_ref, st_ref, it_ref = oracle.icp(kfs[k].depth_f32(), kfs[k].nrm4_f32(), kfs[k].pp, sp, sn, case.sweep,
                                               case.T_init[k][h], prm, max_iters=15)
            dt, dr = synth.pose_error(poses[p], T_ref)
            assert dt < 1e-3 and dr < 1e-4, (p, dt, dr)


def test_autotuner_picks_a_candidate(forest, tmp_path, monkeypatch):
    from paper_2101_00585_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tiles.json"))
    case, prm, sp, sn, kfs = forest
    sw, bufs, batch = _gpu_batch(case, sp, sn, kfs, case.n_hyp)
    res = autotune.tune(batch, _init(case), up.Params(max_iters=3), reps=1)
    assert res["tiles"] in autotune.CANDIDATES and not res["cached"]
    assert len(res["ms"]) == len(autotune.CANDIDATES)
    again = autotune.tune(batch, _init(case), up.Params(max_iters=3))
    assert again["cached"] and again["tiles"] == res["tiles"]


def _check_one_step(case, prm, sp, sn, kfs, recs, poses, p):
    k, h = divmod(p, case.n_hyp)
    Tn, st = oracle.icp_step(kfs[k].depth_f32(), kfs[k].nrm4_f32(), kfs[k].pp, sp, sn, case.sweep,
                             case.T_init[k][h], prm)
    A, A_ref = _upper(recs[p]["A"]), _upper(st["A"])
    assert np.linalg.norm(A - A_ref) <= 1e-5 * np.linalg.norm(A_ref), p
    assert abs(recs[p]["inliers"] - st["inliers"]) <= 2, (p, recs[p]["inliers"], st["inliers"])
    assert recs[p]["valid"] == st["valid"]
    assert recs[p]["status"] == st["status"], p
    if st["status"] == 0:
        dt, dr = synth.pose_error(poses[p], Tn)
        assert dt < 1e-4 and dr < 1e-5, (p, dt, dr)
    return st["status"]


def test_batched_full_size_first_step_matches_oracle(forest_full):
    """All 512 problems of the row's workload, one Gauss-Newton step (the 1.0 m gate), each against the
    oracle's step: J^T J relative 1e-5, inliers within the gate's near-ties, pose 1e-4 m / 1e-5 rad."""
    case, prm, sp, sn, kfs = forest_full
    sw, bufs, batch = _gpu_batch(case, sp, sn, kfs, case.n_hyp)
    assert batch.n_prob == 512
    batch.run(_init(case), up.Params(max_iters=1, **FULL))
    recs = batch.read_stats()
    poses = batch.poses.cpu().numpy().reshape(-1, 3, 4)
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        status = list(ex.map(lambda p: _check_one_step(case, prm, sp, sn, kfs, recs, poses, p), range(512)))
    assert status.count(0) > 400


def test_batched_full_size_registration_matches_oracle(forest_full):
    """The graph-captured launch of all 512 problems (15 steps, coarse-to-fine gate) against the oracle's
    full registration for every hypothesis of one keyframe of each size, at 1e-4 m / 1e-5 rad, with the
    same number of steps."""
    case, prm, sp, sn, kfs = forest_full
    sw, bufs, batch = _gpu_batch(case, sp, sn, kfs, case.n_hyp)
    batch.capture(up.Params(max_iters=15, **FULL))
    batch.init.copy_(_init(case))
    batch.replay()
    recs = batch.read_stats()
    poses = batch.poses.cpu().numpy().reshape(-1, 3, 4)
    picks = [k for k in (0, 22, 43)]
    assert [(kfs[k].pp.rows, kfs[k].pp.cols) for k in picks] == [(256, 1024), (512, 2048), (1024, 4096)]
    jobs = [(k, h) for k in picks for h in range(case.n_hyp)]

    def ref(job):
        k, h = job
        return oracle.icp(kfs[k].depth_f32(), kfs[k].nrm4_f32(), kfs[k].pp, sp, sn, case.sweep, case.T_init[k][h],
                          dataclasses.replace(prm, max_iters=15))

    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        refs = list(ex.map(ref, jobs))
    errs = []
    for (k, h), (T_ref, st_ref, it_ref) in zip(jobs, refs):
        p = k * case.n_hyp + h
        dt, dr = synth.pose_error(poses[p], T_ref)
        errs.append((p, dt, dr, recs[p]["iters"], it_ref))
        assert dt < 1e-4 and dr < 1e-5, errs[-1]
        # the step counts agree, except where one side met the 1e-6 convergence test and the other,
        # its steps hovering at that size as single correspondences flip, ran on (same pose within tolerance)
        if recs[p]["iters"] < it_ref:
            assert recs[p]["converged"] == 1, errs[-1]
        elif recs[p]["iters"] > it_ref:
            assert st_ref["converged"] == 1, errs[-1]
    assert sum(e[3] == e[4] for e in errs) >= 0.75 * len(errs), errs
    print("batched vs oracle (problem, m, rad, steps, oracle steps):", errs)


def test_batched_graph_replay_equals_eager_launch(forest_full):
    """Replaying the captured graph (twice) gives the eager launch's poses and records bit for bit: every
    sum is formed in a fixed order, so a launch does not depend on timing."""
    case, prm, sp, sn, kfs = forest_full
    sw, bufs, batch = _gpu_batch(case, sp, sn, kfs, case.n_hyp)
    p15 = up.Params(max_iters=15, **FULL)
    init = _init(case)
    batch.run(init, p15)
    eager_poses, eager_stats = batch.poses.clone(), batch.stats.clone()
    batch.capture(p15)
    for _ in range(2):
        batch.poses.zero_()
        batch.stats.zero_()
        batch.init.copy_(init)
        batch.replay()
        torch.cuda.synchronize()
        assert torch.equal(batch.poses, eager_poses)
        assert torch.equal(batch.stats, eager_stats)
