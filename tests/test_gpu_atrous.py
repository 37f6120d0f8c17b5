"""GPU parity of the edge-avoiding a-trous normal smoothing (Sec. III-A) against the FP64 oracle.

Tolerance (FP32 path): every tap weight carries a few FP32 roundings plus the error of the
fast exponential (relative <= 2^-21 for the arguments here), the 25-term sums a few more, and
the normalisation one rsqrt: the direction moves by well under 1e-6 rad per level.  The bound
used is 1e-5 rad after up to 5 levels.  FP16 storage rounds every level's output to half
precision (2^-11 relative per component, about 7e-4 rad), so that path is held to 4e-3 rad
after 3 levels.  Validity is copied, so it must match exactly.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from synth import configs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

up = pytest.importorskip("paper_2101_00585_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().float().cpu().numpy()


def _angles(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def _sweep_inputs(cfg):
    if cfg == "room":
        c = configs.room_case(noise=True)
        sc, pp = c.scan, c.sweep
    else:
        seq = configs.tunnel_sequence(n_scans=2)
        sc, pp = seq.scan(1), seq.sweep
    sp4, sn4, _, _ = oracle.sweep_frame(sc, pp, oracle.Params())
    return pp, sp4, sn4


def _compare(pp, sp4, sn4, levels, precision=up.F32, sigma_n=0.5, sigma_x=0.02, tol=1e-5):
    p = up.Params(atrous_levels=levels, atrous_sigma_n=sigma_n, atrous_sigma_x=sigma_x)
    dt = torch.float32 if precision == up.F32 else torch.float16
    nin = dev(sn4).to(dt)
    got = host(up.atrous_normals(dev(sp4), nin, pp, p, precision))
    ref_in = host(nin)  # the oracle smooths exactly what the kernel read
    ref, rv = oracle.atrous(sp4, ref_in[..., :3], ref_in[..., 3] != 0, levels, sigma_n, sigma_x)
    assert np.array_equal(got[..., 3] != 0, rv)
    assert not got[~rv].any()
    ang = _angles(got[rv][:, :3].astype(np.float64), ref[rv])
    assert ang.max() <= tol, (levels, ang.max())
    return ang


@pytest.mark.parametrize("cfg", ["room", "tunnel"])
@pytest.mark.parametrize("levels", [1, 3, 5])
def test_atrous_parity_fp32(cfg, levels):
    pp, sp4, sn4 = _sweep_inputs(cfg)
    _compare(pp, sp4, sn4, levels)


def test_atrous_parity_fp16_storage():
    pp, sp4, sn4 = _sweep_inputs("room")
    _compare(pp, sp4, sn4, 3, up.F16, tol=4e-3)


def test_atrous_sigmas_and_zero_levels():
    pp, sp4, sn4 = _sweep_inputs("room")
    _compare(pp, sp4, sn4, 2, sigma_n=0.2, sigma_x=0.005)
    _compare(pp, sp4, sn4, 2, sigma_n=5.0, sigma_x=1.0)
    got = host(up.atrous_normals(dev(sp4), dev(sn4), pp, up.Params(atrous_levels=0)))
    assert np.array_equal(got, sn4)


def test_atrous_ragged_and_degenerate_images():
    rng = np.random.default_rng(41)
    pp = up_pano(7, 36)
    sp4 = np.zeros((7, 36, 4), np.float32)
    sp4[..., :3] = rng.normal(0, 1, (7, 36, 3)) + np.array([5.0, 0.0, 0.0])
    sp4[..., 3] = 1.0
    n = rng.normal(0, 0.2, (7, 36, 3)) + np.array([-1.0, 0.0, 0.0])
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    valid = rng.random((7, 36)) > 0.3
    sn4 = np.zeros((7, 36, 4), np.float32)
    sn4[valid, :3] = n[valid]
    sn4[valid, 3] = 1.0
    _compare(pp, sp4, sn4, 3)
    # all invalid: output all zeros
    z = np.zeros_like(sn4)
    assert not host(up.atrous_normals(dev(sp4), dev(z), pp, up.Params(atrous_levels=2))).any()
    # one valid pixel keeps its normal
    one = np.zeros_like(sn4)
    one[3, 17] = sn4[valid][0]
    one[3, 17, 3] = 1.0
    got = host(up.atrous_normals(dev(sp4), dev(one), pp, up.Params(atrous_levels=3)))
    assert np.abs(got[3, 17, :3] - one[3, 17, :3]).max() < 1e-6 and got[3, 17, 3] == 1.0


def test_atrous_rejects_bad_arguments():
    import ctypes
    from paper_2101_00585_gb300 import _abi
    pp = up_pano(8, 16)
    L = up.lib()
    ps = up.pano_struct(pp)
    buf = [torch.zeros((8, 16, 4), device="cuda") for _ in range(4)]
    ptr = [ctypes.c_void_p(b.data_ptr()) for b in buf]
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    bad = [_abi.AtrousParams(7, 0.5, 0.02), _abi.AtrousParams(5, 0.5, 0.02), _abi.AtrousParams(2, 0.0, 0.02),
           _abi.AtrousParams(2, 0.5, -1.0), _abi.AtrousParams(-1, 0.5, 0.02)]
    for ap in bad:
        assert L.upslam_atrous_normals(ctypes.byref(ps), ptr[0], ptr[1], ptr[2], ptr[3], up.F32, ctypes.byref(ap),
                                       s) == _abi.ERR_INVALID_ARG
    ok = _abi.AtrousParams(2, 0.5, 0.02)
    # aliasing input and output, missing scratch for two levels
    assert L.upslam_atrous_normals(ctypes.byref(ps), ptr[0], ptr[1], ptr[1], ptr[3], up.F32, ctypes.byref(ok),
                                   s) == _abi.ERR_INVALID_ARG
    assert L.upslam_atrous_normals(ctypes.byref(ps), ptr[0], ptr[1], ptr[2], None, up.F32, ctypes.byref(ok),
                                   s) == _abi.ERR_INVALID_ARG
    assert L.upslam_atrous_normals(ctypes.byref(ps), ptr[0], ptr[1], ptr[2], ptr[3], up.F32, ctypes.byref(ok),
                                   s) == _abi.OK


def test_tracker_with_smoothing_matches_oracle():
    """Workload 2, first 8 sweeps with 3 smoothing levels: the device Tracker vs the oracle's chained path."""
    from tests.helpers import IDENTITY
    import synth
    n = 8
    seq = configs.tunnel_sequence(n_scans=n)
    scans = [seq.scan(k) for k in range(n)]
    prm = oracle.Params(accept_quality=0.1, atrous_levels=3)
    trk = up.Tracker(seq.sweep, seq.kf, up.Params(accept_quality=0.1, atrous_levels=3), constant_velocity=False)
    trk.new_keyframe(dev(scans[0]))
    kf_ref = oracle.Keyframe(seq.kf)
    sp, sn, _, _ = oracle.sweep_frame(scans[0], seq.sweep, prm)
    oracle.fuse(kf_ref, sp, sn, seq.sweep, IDENTITY, prm)
    T_ref = IDENTITY.copy()
    for k in range(1, n):
        trk.track(dev(scans[k]))
        T_ref, st_ref, it_ref, acc_ref = oracle.process_scan(kf_ref, scans[k], seq.sweep, T_ref, prm)
        T = trk.state.pose.cpu().numpy().reshape(3, 4)
        dt, dr = synth.pose_error(T, T_ref)
        assert dt < 1e-3 and dr < 1e-4, (k, dt, dr)
        assert trk.state.read_stats()["accepted"] == int(acc_ref)
    et, er = synth.pose_error(trk.state.pose.cpu().numpy().reshape(3, 4),
                              synth.relative(seq.poses[0], seq.poses[n - 1]))
    assert et < 0.03 and er < math.radians(0.3)


def up_pano(rows, cols):
    from tests.helpers import tiny_pano
    return tiny_pano(rows, cols)
