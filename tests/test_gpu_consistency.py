"""GPU parity of the keyframe mutual consistency check (Sec. III-C): every decision is FP32 with the
same operations on both sides (binning rule, FP32-rounded pose, fixed-order FP64 inverse, the
limit (rel r + abs) + r), so the flags must match the oracle exactly."""
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
from tests.test_gpu_parity import dev, pose_dev  # noqa: E402
from tests.test_oracle_consistency_pins import _room_pair  # noqa: E402


def _kf(depth, pp, precision=up.F32):
    kf = up.KeyframeBuffer(pp, "cuda", precision)
    nw = np.zeros(depth.shape + (4,), np.float32)
    nw[..., 2] = 1.0
    nw[..., 3] = (depth > 0).astype(np.float32)
    kf.set(dev(depth), dev(nw).to(kf.nw.dtype))
    return kf


def _run(da, pa, db, pb, T_ab, precision=up.F32, rel=0.05, abs_m=0.2):
    ka, kb = _kf(da, pa, precision), _kf(db, pb, precision)
    removed, fa, fb = up.keyframe_consistency(ka, kb, pose_dev(T_ab), rel, abs_m)
    torch.cuda.synchronize()
    ra, rb = oracle.consistency(da, pa, db, pb, T_ab, rel, abs_m)
    assert np.array_equal(fa.cpu().numpy().astype(bool), ra)
    assert np.array_equal(fb.cpu().numpy().astype(bool), rb)
    assert removed.cpu().tolist() == [int(ra.sum()), int(rb.sum())]
    # flagged samples are emptied, the rest untouched
    assert np.array_equal(ka.depth.cpu().numpy(), np.where(ra, 0.0, da).astype(np.float32))
    assert np.array_equal(kb.depth.cpu().numpy(), np.where(rb, 0.0, db).astype(np.float32))
    assert not ka.nw.float().cpu().numpy()[ra].any()
    return ra, rb


@pytest.mark.parametrize("box", [False, True])
def test_consistency_room_exact(box):
    kp, da, db, T_ab, ida, n_static = _room_pair(box)
    ra, rb = _run(da, kp, db, kp, T_ab)
    if box:
        assert ra.sum() > 4000 and rb.sum() == 0
    else:
        assert ra.sum() == 0 and rb.sum() == 0


def test_consistency_fp16_storage_same_flags():
    kp, da, db, T_ab, _, _ = _room_pair(True)
    _run(da, kp, db, kp, T_ab, precision=up.F16)


def test_consistency_full_size_tunnel_keyframes():
    """Two 512 x 2048 keyframes rendered in the tunnel 10 sweeps (1 m) apart; then a patch of the first
    one pulled 40 % closer (an object that has since left)."""
    seq = configs.tunnel_sequence(n_scans=12)
    kfs = [synth.render_keyframe(seq.scene, seq.kf, seq.poses[k])[0].astype(np.float32) for k in (0, 10)]
    T_ab = synth.relative(seq.poses[0], seq.poses[10])
    ra, rb = _run(kfs[0], seq.kf, kfs[1], seq.kf, T_ab)
    assert ra.sum() <= 1e-3 * (kfs[0] > 0).sum() and rb.sum() <= 1e-3 * (kfs[1] > 0).sum()
    # a rectangle of A's samples pulled 40 % closer (a "vehicle" that has since left)
    da = kfs[0].copy()
    da[200:260, 900:1100] = np.where(da[200:260, 900:1100] > 0, 0.6 * da[200:260, 900:1100], 0)
    ra, _ = _run(da, seq.kf, kfs[1], seq.kf, T_ab)
    assert ra[200:260, 900:1100].sum() > 0.5 * (da[200:260, 900:1100] > 0).sum()


def test_consistency_rejects_bad_arguments():
    from paper_2101_00585_gb300 import _abi
    kp, da, db, T_ab, _, _ = _room_pair(False)
    ka = _kf(da, kp)
    L = up.lib()
    s = ka.struct()
    ws = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    T = pose_dev(T_ab)
    assert L.upslam_keyframe_consistency(ctypes.byref(s), ctypes.byref(s), ctypes.c_void_p(T.data_ptr()), 0.05, 0.2,
                                         ctypes.c_void_p(ws.data_ptr()), ws.numel(), None, None) == _abi.ERR_INVALID_ARG
    kb = _kf(db, kp)
    sb = kb.struct()
    assert L.upslam_keyframe_consistency(ctypes.byref(s), ctypes.byref(sb), ctypes.c_void_p(T.data_ptr()), -1.0, 0.2,
                                         ctypes.c_void_p(ws.data_ptr()), ws.numel(), None, None) == _abi.ERR_INVALID_ARG
    assert L.upslam_keyframe_consistency(ctypes.byref(s), ctypes.byref(sb), ctypes.c_void_p(T.data_ptr()), 0.05, 0.2,
                                         ctypes.c_void_p(ws.data_ptr()), 16, None, None) == _abi.ERR_INVALID_ARG


def test_tracker_switch_with_consistency():
    seq = configs.tunnel_sequence(n_scans=8)
    trk = up.Tracker(seq.sweep, seq.kf, up.Params(accept_quality=0.1))
    pool = [up.KeyframeBuffer(seq.kf) for _ in range(2)]
    trk.new_keyframe(dev(seq.scan(0)))
    for k in range(1, 6):
        trk.track(dev(seq.scan(k)))
    trk.new_keyframe(buffer=pool[0], consistency=True)
    for k in range(6, 8):
        trk.track(dev(seq.scan(k)))
    torch.cuda.synchronize()
    removed = trk.last_removed.cpu().tolist()
    assert removed[0] <= 1e-3 * 1048576 and removed[1] <= 1e-3 * 1048576
    et, er = synth.pose_error(trk.state.pose.cpu().numpy().reshape(3, 4), synth.relative(seq.poses[5], seq.poses[7]))
    assert et < 0.03 and er < math.radians(0.3)
