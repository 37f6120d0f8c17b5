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

import math

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


@pytest.fixture(scope="module")
def forest():
    case = configs.forest_batch(n_kf=len(SIZES), n_hyp=4, max_trans=0.3, max_rot_deg=3.0, kf_sizes=SIZES)
    prm = oracle.Params()
    sp, sn, _, _ = oracle.sweep_frame(case.scan, case.sweep, prm)
    kfs = []
    for i, (P_kf, kp) in enumerate(zip(case.kf_poses, case.kf_panos)):
        sc = synth.scan(case.scene, case.lidar, P_kf, np.random.default_rng((4, 100 + i)))
        kp_sweep, kn_sweep, _, _ = oracle.sweep_frame(sc, case.sweep, prm)
        kf = oracle.Keyframe(kp)
        oracle.fuse(kf, kp_sweep, kn_sweep, case.sweep, IDENTITY, prm)
        kfs.append(kf)
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
