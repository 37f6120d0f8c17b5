"""Precision form (workload 3): FP16 normals and sample counts, FP32 depth.

Workload 3: 128 x 2048 campus sweeps, 1024 x 4096 keyframes.  The kernels read FP16 normals and counts,
accumulate J^T J / J^T r in FP32 with compensated CTA and cross-CTA sums, and solve in FP64.

The oracle receives the same FP16-rounded values, converted exactly to FP32, so parity is checked at the
same tolerances as the FP32 path:
* poses: 1e-4 m and 1e-5 rad;
* J^T J: relative 1e-5;
* hole-fill winners: exact.

The cost of FP16 storage itself is measured separately: the FP16 registration against the FP32 one on the
unrounded inputs.  It stays within 2 mm / 0.01 deg, far below the 2 cm sensor noise.
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


def _f16(a):
    return np.asarray(a, np.float32).astype(np.float16).astype(np.float32)


@pytest.fixture(scope="module")
def campus():
    """Oracle keyframe from two campus sweeps, and a third sweep frame to register."""
    seq = configs.campus_sequence(n_scans=4)
    prm = oracle.Params(accept_quality=0.1)
    kf = oracle.Keyframe(seq.kf)
    sp0, sn0, _, _ = oracle.sweep_frame(seq.scan(0), seq.sweep, prm)
    oracle.fuse(kf, sp0, sn0, seq.sweep, IDENTITY, prm)
    sp1, sn1, _, _ = oracle.sweep_frame(seq.scan(1), seq.sweep, prm)
    oracle.fuse(kf, sp1, sn1, seq.sweep, synth.relative(seq.poses[0], seq.poses[1]), prm)
    sp2, sn2, _, _ = oracle.sweep_frame(seq.scan(2), seq.sweep, prm)
    return seq, prm, kf, sp2, sn2


def _buffers(seq, kd, kn, sp, sn, precision):
    dt = torch.float32 if precision == up.F32 else torch.float16
    kf = up.KeyframeBuffer(seq.kf, "cuda", precision)
    kf.set(torch.from_numpy(kd).cuda(), torch.from_numpy(kn).cuda().to(dt))
    sw = up.SweepFrame(seq.sweep, "cuda", precision)
    sw.set(torch.from_numpy(sp).cuda(), torch.from_numpy(sn).cuda().to(dt))
    return kf, sw


def _upper(a):
    A = np.zeros((6, 6))
    A[np.triu_indices(6)] = a
    return A + np.triu(A, 1).T


def test_precision_form_icp_parity_and_storage_cost(campus):
    seq, prm, kf_ref, sp, sn = campus
    kd, kn = kf_ref.depth_f32(), kf_ref.nrm4_f32()
    kn16, sn16 = _f16(kn), _f16(sn)
    T0 = synth.relative(seq.poses[0], seq.poses[1])
    # one step: normal equations against the oracle on identical (FP16-rounded) inputs
    kf, sw = _buffers(seq, kd, kn16, sp, sn16, up.F16)
    st1 = up.IcpState(kf)
    st1.pose.copy_(torch.from_numpy(T0.reshape(12).copy()).cuda())
    up.icp(kf, sw, st1, up.Params(max_iters=1))
    rec = st1.read_stats()
    ne = oracle.normal_equations(kd, kn16, seq.kf, sp, sn16, seq.sweep, T0, prm)
    A, A_ref = _upper(rec["A"]), _upper(ne["A"])
    assert np.linalg.norm(A - A_ref) <= 1e-5 * np.linalg.norm(A_ref)
    # full registration
    st = up.IcpState(kf)
    st.pose.copy_(torch.from_numpy(T0.reshape(12).copy()).cuda())
    up.icp(kf, sw, st, up.Params(max_iters=15))
    T16 = st.pose.cpu().numpy().reshape(3, 4)
    T_ref, _, it_ref = oracle.icp(kd, kn16, seq.kf, sp, sn16, seq.sweep, T0, prm)
    dt, dr = synth.pose_error(T16, T_ref)
    assert dt < 1e-4 and dr < 1e-5, (dt, dr)
    assert st.read_stats()["iters"] == it_ref
    # cost of the storage precision: FP16 vs FP32 registration on the unrounded inputs
    kf32, sw32 = _buffers(seq, kd, kn, sp, sn, up.F32)
    s32 = up.IcpState(kf32)
    s32.pose.copy_(torch.from_numpy(T0.reshape(12).copy()).cuda())
    up.icp(kf32, sw32, s32, up.Params(max_iters=15))
    et, er = synth.pose_error(T16, s32.pose.cpu().numpy().reshape(3, 4))
    print(f"\nprecision form: FP16-vs-oracle {dt:.2e} m {dr:.2e} rad; FP16-vs-FP32 storage {et:.2e} m "
          f"{math.degrees(er):.2e} deg; J^T J rel {np.linalg.norm(A - A_ref) / np.linalg.norm(A_ref):.2e}")
    assert et < 2e-3 and er < math.radians(0.01)


def test_precision_form_fusion_parity(campus):
    seq, prm, kf_ref, sp, sn = campus
    kd, kn = kf_ref.depth_f32(), kf_ref.nrm4_f32()
    kn16, sn16 = _f16(kn), _f16(sn)
    T = synth.relative(seq.poses[0], seq.poses[2])
    kf, sw = _buffers(seq, kd, kn16, sp, sn16, up.F16)
    up.fuse(kf, sw, torch.from_numpy(T.reshape(12).copy()).cuda(), up.Params(), None)
    ref = oracle.Keyframe(seq.kf, kd.astype(np.float64), kn16[..., :3].astype(np.float64), kn16[..., 3].astype(np.float64))
    fused, filled = oracle.fuse(ref, sp, sn16, seq.sweep, T, prm)
    gd = kf.depth.cpu().numpy().astype(np.float64)
    gn = kf.nw.float().cpu().numpy().astype(np.float64)
    wdiff = gn[..., 3] != ref.w
    assert wdiff.sum() <= max(2, 1e-4 * (ref.w > 0).sum())
    same = ~wdiff & (ref.w > 0)
    # depth is FP32 in both forms
    assert np.allclose(gd[same], ref.depth[same], rtol=2e-6, atol=0)
    # normals are stored in FP16: 2^-11 per component
    a = gn[..., :3][same]
    b = ref.nrm[same]
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    ang = np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), (a * b).sum(-1))
    assert ang.max() <= 2e-3
    assert fused > 1000 and filled > 1000
