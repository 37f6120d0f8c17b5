"""GPU parity of the loop-closure grid search (Sec. III-C) against the oracle, and its use.

Scores are inlier counts.  Bins are bit-exact on both sides (the FP32 rule); the two gates of
Omega are FP32 on the device and FP64 in the oracle, so a count may differ by the handful of
near-ties the ICP parity tests allow (<= 3 here).  The winner must be a candidate whose oracle
score is within that margin of the oracle's best.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import pytest

import oracle
import synth
from synth import configs
from tests.helpers import IDENTITY, room_sweep_and_keyframe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

up = pytest.importorskip("paper_2101_00585_gb300")
from tests.test_gpu_parity import _kf_buffers, _sweep_buffers, dev, pose_dev, pose_host, rot_err  # noqa: E402

TIE = 3


def _grid_twists(n_xy=5, n_yaw=5, step=0.1, yaw_step_deg=2.0):
    out = []
    h = (n_xy - 1) / 2
    hy = (n_yaw - 1) / 2
    for i in range(n_xy):
        for j in range(n_xy):
            for k in range(n_yaw):
                out.append([0.0, 0.0, math.radians((k - hy) * yaw_step_deg), (i - h) * step, (j - h) * step, 0.0])
    return np.array(out, np.float32)


def _host_poses(center, xi):
    return np.stack([oracle.se3_exp_left(x.astype(np.float64), center).reshape(12) for x in xi])


def _check(scores, best, ref_scores):
    s = scores.cpu().numpy()
    assert np.abs(s - ref_scores).max() <= TIE, np.abs(s - ref_scores).max()
    b = int(best.cpu().numpy()[0])
    assert s[b] == s.max() and b == int(np.argmax(s))
    assert ref_scores[b] >= ref_scores.max() - 2 * TIE


@pytest.mark.parametrize("stride", [1, 2, 4])
def test_grid_score_parity_workload1(stride):
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    p = oracle.Params(d_max=0.1)
    center = synth.perturb(c.T_true, np.random.default_rng(81), 0.05, 0.02)
    poses = _host_poses(center, _grid_twists())
    ref, ref_best = oracle.grid_score(kd, kn, c.kf, sp4, sn4, c.sweep, poses, stride, p)
    kf, sw = _kf_buffers(kd, kn, c.kf), _sweep_buffers(sp4, sn4, c.sweep)
    scores, best, best_pose = up.grid_score(kf, sw, dev(poses), up.Params(d_max=0.1), stride)
    _check(scores, best, ref)
    b = int(best.cpu()[0])
    assert np.array_equal(best_pose.cpu().numpy(), poses[b])


def test_grid_score_full_size_sampled():
    """512 x 2048 keyframe, 64 x 1024 sweep, 200 candidates at stride 4; 12 candidates checked by the oracle."""
    seq = configs.tunnel_sequence(n_scans=3)
    prm = oracle.Params(accept_quality=0.1, d_max=0.2)
    kf_ref = oracle.Keyframe(seq.kf)
    sp0, sn0, _, _ = oracle.sweep_frame(seq.scan(0), seq.sweep, prm)
    oracle.fuse(kf_ref, sp0, sn0, seq.sweep, IDENTITY, prm)
    sp4, sn4, _, _ = oracle.sweep_frame(seq.scan(2), seq.sweep, prm)
    kd, kn = kf_ref.depth_f32(), kf_ref.nrm4_f32()
    center = synth.relative(seq.poses[0], seq.poses[2])
    xi = _grid_twists(n_xy=5, n_yaw=8)
    poses = _host_poses(center, xi)
    kf, sw = _kf_buffers(kd, kn, seq.kf), _sweep_buffers(sp4, sn4, seq.sweep)
    scores, best, _ = up.grid_score(kf, sw, dev(poses), up.Params(d_max=0.2), 4)
    s = scores.cpu().numpy()
    pick = np.random.default_rng(82).choice(len(poses), 12, replace=False)
    ref, _ = oracle.grid_score(kd, kn, seq.kf, sp4, sn4, seq.sweep, poses[pick], 4, prm)
    assert np.abs(s[pick] - ref).max() <= TIE
    assert int(best.cpu()[0]) == int(np.argmax(s))


def test_grid_score_batch_equals_single_candidates():
    """Each lane of a CTA scores its own candidate: a batch of 75 distinct candidates (two full CTA rows of
    32 and a ragged 11) gives every candidate exactly the count it gets alone, at full keyframe size and on
    the room, FP32 and FP16 keyframe storage."""
    seq = configs.tunnel_sequence(n_scans=3)
    prm = oracle.Params(accept_quality=0.1, d_max=0.2)
    kf_ref = oracle.Keyframe(seq.kf)
    sp0, sn0, _, _ = oracle.sweep_frame(seq.scan(0), seq.sweep, prm)
    oracle.fuse(kf_ref, sp0, sn0, seq.sweep, IDENTITY, prm)
    sp4, sn4, _, _ = oracle.sweep_frame(seq.scan(2), seq.sweep, prm)
    kd, kn = kf_ref.depth_f32(), kf_ref.nrm4_f32()
    c, _, rsp4, rsn4, rkd, rkn = room_sweep_and_keyframe(noise=True)
    cases = [(kd, kn, seq.kf, sp4, sn4, seq.sweep, synth.relative(seq.poses[0], seq.poses[2]), 4, up.F32),
             (rkd, rkn, c.kf, rsp4, rsn4, c.sweep, c.T_true, 2, up.F16)]
    for kd_, kn_, kpp, sp_, sn_, spp, center, stride, prec in cases:
        kf, sw = _kf_buffers(kd_, kn_, kpp, prec), _sweep_buffers(sp_, sn_, spp)
        xi = _grid_twists(n_xy=5, n_yaw=3, step=0.05, yaw_step_deg=1.0)  # 75 candidates
        poses = dev(_host_poses(center, xi))
        scores, _, _ = up.grid_score(kf, sw, poses, up.Params(d_max=0.2), stride)
        s = scores.cpu().numpy()
        assert s.max() > 0
        for i in range(poses.shape[0]):
            one, _, _ = up.grid_score(kf, sw, poses[i:i + 1].contiguous(), up.Params(d_max=0.2), stride)
            assert int(one.cpu()[0]) == int(s[i]), (i, int(one.cpu()[0]), int(s[i]))


def test_grid_candidates_match_host_composition():
    center = synth.perturb(IDENTITY, np.random.default_rng(83), 1.0, 0.3)
    xi = np.random.default_rng(84).normal(0, 0.3, (37, 6)).astype(np.float32)
    got = up.grid_candidates(pose_dev(center), dev(xi)).cpu().numpy()
    ref = _host_poses(center, xi)
    assert np.abs(got - ref).max() < 1e-13


def test_grid_edge_cases():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf, sw = _kf_buffers(kd, kn, c.kf), _sweep_buffers(sp4, sn4, c.sweep)
    p = up.Params(d_max=0.1)
    # identical candidates: equal scores, the first one wins; a ragged count (13, fewer than one CTA's 32)
    poses = np.stack([c.T_true.reshape(12)] * 13)
    scores, best, _ = up.grid_score(kf, sw, dev(poses), p, 3)
    s = scores.cpu().numpy()
    assert (s == s[0]).all() and s[0] > 0 and int(best.cpu()[0]) == 0
    # one candidate; a stride wider than the image samples pixel (0, 0) only
    one = dev(c.T_true.reshape(1, 12))
    scores, best, _ = up.grid_score(kf, sw, one, p, 10_000)
    assert int(best.cpu()[0]) == 0 and int(scores.cpu()[0]) <= 1
    # an empty keyframe scores zero everywhere
    empty = _kf_buffers(np.zeros_like(kd), np.zeros_like(kn), c.kf)
    scores, best, _ = up.grid_score(empty, sw, dev(poses[:5]), p, 2)
    assert not scores.cpu().numpy().any() and int(best.cpu()[0]) == 0
    # bad arguments
    from paper_2101_00585_gb300 import _abi
    L = up.lib()
    ks, ss, ip = kf.struct(), sw.struct(), p.icp()
    buf = torch.zeros(64, dtype=torch.int64, device="cuda")
    for n, stride in ((0, 2), (5, 0), (-1, 2)):
        assert L.upslam_grid_score(ctypes.byref(ks), ctypes.byref(ss), ctypes.c_void_p(one.data_ptr()), n, stride,
                                   ctypes.byref(ip), ctypes.c_void_p(buf.data_ptr()),
                                   ctypes.c_void_p(buf.data_ptr() + 256), None, None) == _abi.ERR_INVALID_ARG


def test_grid_search_then_icp_recovers_a_large_offset():
    """A start 0.35 m / 6 deg off: plain ICP from it vs grid search (promoted to ICP) on the room."""
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf, sw = _kf_buffers(kd, kn, c.kf), _sweep_buffers(sp4, sn4, c.sweep)
    off = synth.pose(synth.rot_zyx(math.radians(6.0)), [0.3, -0.2, 0.0])
    start = synth.pose_mul(off, c.T_true)
    xi = _grid_twists(n_xy=9, n_yaw=9, step=0.1, yaw_step_deg=2.0)  # 729 candidates, +-0.4 m, +-8 deg
    poses = up.grid_candidates(pose_dev(start), dev(xi))
    scores, best, best_pose = up.grid_score(kf, sw, poses, up.Params(d_max=0.1), 4)
    state = up.IcpState(kf)
    state.pose.copy_(best_pose)
    up.icp(kf, sw, state, up.Params(max_iters=30))
    et, er = rot_err(pose_host(state.pose), c.T_true)
    assert et < 0.01 and er < math.radians(0.1), (et, er)
