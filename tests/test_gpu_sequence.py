"""GPU parity of the motion prior and of the benchmark's per-sweep launch against the FP64 oracle.

The benchmark registers every sweep with ``upslam_track_scan`` (projection,
normals, the zero-acceleration prior of the Sec. IV-F footnote, ICP of
Sec. III-B and the keyframe update of Sec. III-C in one launch).  These tests
check that exact form:

* the prior's entry points against ``oracle.predict_pose`` / ``update_motion``;
* each sweep of a tunnel sequence started from the oracle's own state (keyframe,
  previous pose, last motion): pose within 1e-4 m / 1e-5 rad, the motion and
  previous-pose outputs, the acceptance decision, and the keyframe it leaves
  against the oracle's keyframe update at the registered pose;
* the whole chained sequence, device state carried from sweep to sweep, at the
  same bound.
"""
from __future__ import annotations

import ctypes
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pose_dev(T):
    return dev(np.ascontiguousarray(T, np.float64).reshape(12))


def pose_host(t):
    return t.detach().cpu().numpy().reshape(3, 4)


def _random_pose(rng, rot=1.0, trans=2.0):
    xi = np.r_[rng.standard_normal(3) * rot, rng.standard_normal(3) * trans]
    return oracle.se3_exp_left(xi, IDENTITY)


def test_motion_prior_entry_points_match_oracle():
    """upslam_predict_pose / upslam_update_motion (FP64 on the device) against the oracle's plain FP64
    product, inverse and Gram-Schmidt, within 1e-14; the zero-velocity prior copies T_prev exactly."""
    L = up.lib()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(71)
    for _ in range(16):
        A, B = _random_pose(rng), _random_pose(rng)
        # a drifted motion: rows scaled and skewed, as rounding would leave it after many products
        M = _random_pose(rng, 0.05, 0.2)
        M[:, :3] = M[:, :3] * (1 + 1e-7 * rng.standard_normal((3, 1))) + 1e-7 * rng.standard_normal((3, 3))
        dA, dB, dM = pose_dev(A), pose_dev(B), pose_dev(M)
        out = torch.empty(12, dtype=torch.float64, device="cuda")
        assert L.upslam_predict_pose(ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dM.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), s) == 0
        assert np.abs(pose_host(out) - oracle.predict_pose(A, M)).max() < 1e-14
        assert L.upslam_predict_pose(ctypes.c_void_p(dA.data_ptr()), None, ctypes.c_void_p(out.data_ptr()), s) == 0
        assert np.array_equal(pose_host(out), A)
        assert L.upslam_update_motion(ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), s) == 0
        assert np.abs(pose_host(out) - oracle.update_motion(A, B)).max() < 1e-14
    # in place (d_T_out aliases d_T_prev)
    A, M = _random_pose(rng), _random_pose(rng, 0.05, 0.2)
    dA, dM = pose_dev(A), pose_dev(M)
    assert L.upslam_predict_pose(ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dM.data_ptr()),
                                 ctypes.c_void_p(dA.data_ptr()), s) == 0
    assert np.abs(pose_host(dA) - oracle.predict_pose(A, M)).max() < 1e-14


def _first_keyframe(seq, scan0, prm):
    kf_ref = oracle.Keyframe(seq.kf)
    sp, sn, _, _ = oracle.sweep_frame(scan0, seq.sweep, prm)
    oracle.fuse(kf_ref, sp, sn, seq.sweep, IDENTITY, prm)
    return kf_ref


@pytest.mark.parametrize("constant_velocity", [True, False])
def test_track_scan_resynchronised_per_sweep(constant_velocity):
    """Every sweep of a 12-sweep tunnel sequence, each started from the oracle's state: the one-launch
    form with the motion prior equals the oracle's prior -> ICP -> motion update -> keyframe update."""
    n = 12
    seq = configs.tunnel_sequence(n_scans=n)
    scans = [seq.scan(k) for k in range(n)]
    prm = oracle.Params(accept_quality=0.1)
    trk = up.Tracker(seq.sweep, seq.kf, up.Params(accept_quality=0.1), constant_velocity=constant_velocity)
    assert trk.front_fused and trk.launches_per_track == 1
    kf_ref = _first_keyframe(seq, scans[0], prm)
    T_prev, M = IDENTITY.copy(), IDENTITY.copy()
    worst = (0.0, 0.0)
    for k in range(1, n):
        kd32, kn32 = kf_ref.depth_f32(), kf_ref.nrm4_f32()
        trk.kf.set(dev(kd32), dev(kn32))
        trk.prev.copy_(pose_dev(T_prev))
        trk.motion.copy_(pose_dev(M))
        trk.track(dev(scans[k]))
        T_ref, st_ref, it_ref, acc_ref, M_ref = oracle.track(kf_ref, scans[k], seq.sweep, T_prev, M, prm,
                                                             constant_velocity)
        st = trk.state.read_stats()
        dt, dr = synth.pose_error(pose_host(trk.state.pose), T_ref)
        worst = (max(worst[0], dt), max(worst[1], dr))
        assert dt < 1e-4 and dr < 1e-5, (k, dt, dr)
        # step counts agree, except where one side met the 1e-6 convergence test while the other's steps
        # hovered at that size (the poses then agree within the bound above)
        if st["iters"] != it_ref:
            assert (st["converged"] if st["iters"] < it_ref else st_ref["converged"]) == 1, (k, st["iters"], it_ref)
        assert st["accepted"] == int(acc_ref)
        assert np.abs(pose_host(trk.prev) - pose_host(trk.state.pose)).max() == 0
        mt, mr = synth.pose_error(pose_host(trk.motion), M_ref)
        assert mt < 1e-4 and mr < 1e-5, (k, mt, mr)
        # the keyframe it leaves equals the oracle's keyframe update of the same FP32 state at the pose
        # the launch registered (a 1e-5 m pose difference moves whole pixel bins): sample counts equal
        # except at gate near-ties, depths to FP32 rounding
        ref = oracle.Keyframe(seq.kf, kd32.astype(np.float64), kn32[..., :3].astype(np.float64),
                              kn32[..., 3].astype(np.float64))
        if acc_ref:
            sp, sn, _, _ = oracle.sweep_frame(scans[k], seq.sweep, prm)
            oracle.fuse(ref, sp, sn, seq.sweep, pose_host(trk.state.pose), prm)
        gw = trk.kf.nw[..., 3].cpu().numpy().astype(np.float64)
        diff = gw != ref.w
        assert diff.sum() <= max(3, 1e-4 * (ref.w > 0).sum()), (k, int(diff.sum()))
        same = ~diff & (ref.w > 0)
        gd = trk.kf.depth.cpu().numpy().astype(np.float64)
        assert np.allclose(gd[same], ref.depth[same], rtol=2e-6, atol=0), k
        T_prev, M = T_ref, M_ref
    print("resynchronised worst pose error", worst)


@pytest.mark.parametrize("constant_velocity", [True, False])
def test_track_scan_chained_sequence(constant_velocity):
    """The benchmark's form chained over 12 tunnel sweeps, every state (keyframe, previous pose, motion)
    carried on the device as the benchmark carries it, against the oracle's chained sequence: each
    registered pose within 1e-4 m / 1e-5 rad, the same acceptance, and within 3 cm / 0.3 deg of the
    truth at the end."""
    n = 12
    seq = configs.tunnel_sequence(n_scans=n)
    scans = [seq.scan(k) for k in range(n)]
    prm = oracle.Params(accept_quality=0.1)
    trk = up.Tracker(seq.sweep, seq.kf, up.Params(accept_quality=0.1), constant_velocity=constant_velocity)
    trk.new_keyframe(dev(scans[0]))
    kf_ref = _first_keyframe(seq, scans[0], prm)
    T_prev, M = IDENTITY.copy(), IDENTITY.copy()
    errs = []
    for k in range(1, n):
        trk.track(dev(scans[k]))
        T_prev_next, st_ref, it_ref, acc_ref, M = oracle.track(kf_ref, scans[k], seq.sweep, T_prev, M, prm,
                                                               constant_velocity)
        T_prev = T_prev_next
        dt, dr = synth.pose_error(pose_host(trk.state.pose), T_prev)
        errs.append((dt, dr))
        assert dt < 1e-4 and dr < 1e-5, (k, errs)
        assert trk.state.read_stats()["accepted"] == int(acc_ref)
    print("chained pose errors", errs)
    et, er = synth.pose_error(pose_host(trk.state.pose), synth.relative(seq.poses[0], seq.poses[n - 1]))
    assert et < 0.03 and er < math.radians(0.3)
