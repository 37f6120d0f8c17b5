"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Inputs are seeded synthetic scans from ``synth`` and intermediate arrays
produced by the oracle; the CUDA library only ever computes the outputs under
test.  Tolerances:

* pixel bins, z-buffer winners, direction tables, hole-fill winners: bit-exact
  (integer decisions taken with the same FP32 operations on both sides);
* similarity-gate and normal-validity decisions: identical except at near-ties,
  where the FP64 margin to the threshold is below the FP32 rounding of the
  tested quantity;
* J^T J: relative Frobenius error <= 1e-5; poses: 1e-4 m and 1e-5 rad;
* depths: relative 2e-6 (FP32 storage of an FP64 result, a few roundings);
  normals: an angle bound from the conditioning of the cross product (see
  ``_normals_compare``).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synth
from synth import configs
from tests.helpers import IDENTITY, room_sweep_and_keyframe, tiny_pano

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

up = pytest.importorskip("paper_2101_00585_gb300")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def pose_dev(T):
    return dev(np.ascontiguousarray(T, np.float64).reshape(12))


def pose_host(t):
    return host(t).reshape(3, 4)


def rot_err(A, B):
    return synth.pose_error(A, B)


def angle_between(a, b):
    """Angle between direction vectors, well conditioned near 0 (normalise in FP64, then atan2)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), (a * b).sum(-1))


# ----------------------------------------------------------------------------- a1


# every panorama geometry the five workloads use: sweeps 16x512, 64x1024, 128x2048; keyframes 256x512,
# 256x1024, 512x2048, 1024x4096; the 64x256 network-input keyframe; and a ragged tiny one
_PANOS = {"sweep16": lambda: configs.LIDAR_16.pano(), "sweep64": lambda: configs.LIDAR_64.pano(),
          "sweep128": lambda: configs.LIDAR_128.pano(), "kf256x512": lambda: synth.keyframe_pano(256, 512),
          "room_kf256x512": lambda: configs.room_case().kf,
          "kf256x1024": lambda: synth.keyframe_pano(256, 1024, 0.3, 150.0),
          "kf512x2048": lambda: synth.keyframe_pano(512, 2048, 0.3, 150.0),
          "kf1024x4096": lambda: synth.keyframe_pano(1024, 4096, 0.3, 150.0),
          "kf64x256": lambda: synth.keyframe_pano(64, 256, 0.3, 150.0),
          "kf128x512": lambda: synth.keyframe_pano(128, 512, 0.3, 30.0), "tiny": lambda: tiny_pano(3, 5)}


@pytest.mark.parametrize("pano", sorted(_PANOS))
def test_direction_table_bit_exact(pano):
    """FP64 sincos on the device rounded to FP32 against the oracle's libm cos/sin rounded to FP32: every
    binning decision that uses a pixel's direction rests on these bits."""
    pp = _PANOS[pano]()
    got = host(up.pano_dirs(pp))
    rt, ct = oracle.dir_table(pp)
    assert np.array_equal(got.view(np.uint32), np.concatenate([rt, ct]).view(np.uint32))


def _assert_project_equal(pts, pp, T=None):
    d_ref, i_ref = oracle.project(pts, pp, T)
    d, i, pix = up.project(dev(pts), pp, None if T is None else pose_dev(T))
    torch.cuda.synchronize()
    assert np.array_equal(host(i), i_ref)
    assert np.array_equal(host(d).view(np.uint32), d_ref.view(np.uint32))
    P = host(pix)
    m = i_ref >= 0
    assert np.array_equal(P[m, :3], pts[i_ref[m], :3]) and np.all(P[m, 3] == 1) and np.all(P[~m] == 0)


def test_project_workload1_bit_exact():
    c = configs.room_case(noise=True)
    _assert_project_equal(c.scan, c.sweep)
    _assert_project_equal(c.scan, c.kf, c.T_true)


def test_project_workload2_full_size_bit_exact():
    seq = configs.tunnel_sequence(n_scans=4)
    sc = seq.scan(3)
    _assert_project_equal(sc, seq.sweep)
    T = synth.relative(seq.poses[0], seq.poses[3])
    _assert_project_equal(sc, seq.kf, T)


def _workload_projection_cases():
    """(name, scan, panorama, pose or None) for the other workloads' sweeps and keyframe scatters: the campus
    128 x 2048 sweep and its 1024 x 4096 keyframe a few sweeps on; the forest sweep binned into each keyframe
    size of the batch at a 2 m / 20 deg hypothesis; a road pair of the learned form."""
    out = []
    camp = configs.campus_sequence(n_scans=4)
    sc = camp.scan(3)
    out.append(("campus sweep", sc, camp.sweep, None))
    out.append(("campus keyframe", sc, camp.kf, synth.relative(camp.poses[0], camp.poses[3])))
    case = configs.forest_batch(n_kf=3, n_hyp=1, kf_sizes=((256, 1024), (512, 2048), (1024, 4096)))
    out.append(("forest sweep", case.scan, case.sweep, None))
    for k in range(3):
        out.append((f"forest keyframe {k}", case.scan, case.kf_panos[k], case.T_init[k][0]))
    road = synth.road(20210105)
    lid = configs.LIDAR_64
    P = synth.pose(synth.rot_zyx(0.3, 0.0, 0.0), [2.0, 0.5, 1.8])
    rs = synth.scan(road, lid, P, np.random.default_rng(5))
    out.append(("road sweep", rs, lid.pano(), None))
    out.append(("road keyframe", rs, synth.keyframe_pano(512, 2048, 0.3, 150.0),
                synth.perturb(IDENTITY, np.random.default_rng(6), 1.0, math.radians(30.0))))
    return out


def test_project_bit_exact_on_every_workload():
    """Pixel winners and depths bit for bit against the oracle for the sweeps and keyframe scatters of
    workloads 3 to 5 (workloads 1 and 2 above), and the sweep normals of the campus form within the
    conditioning bound, in FP32 and FP16 storage."""
    for name, sc, pp, T in _workload_projection_cases():
        _assert_project_equal(sc, pp, T)
    camp = configs.campus_sequence(n_scans=2)
    depth, idx = oracle.project(camp.scan(1), camp.sweep)
    pix = oracle.pixel_points(camp.scan(1), idx)
    assert _normals_compare(pix, depth, camp.sweep) > 0.8 * (idx >= 0).sum()
    _normals_compare(pix, depth, camp.sweep, up.F16)


def test_project_collisions_ragged_and_empty():
    """Many points per pixel (z-buffer ties), odd sizes, no points, all invalid."""
    pp = tiny_pano(8, 16)
    rng = np.random.default_rng(21)
    for n in (1, 7, 255, 257, 4099):
        pts = np.zeros((n, 4), np.float32)
        pts[:, :3] = rng.standard_normal((n, 3)) * 3
        pts[:, 3] = (rng.random(n) < 0.9).astype(np.float32)
        pts[n // 2:, :3] = pts[: n - n // 2, :3]  # exact duplicates: ties broken by index
        _assert_project_equal(pts, pp)
    _assert_project_equal(np.zeros((0, 4), np.float32), pp)
    _assert_project_equal(np.zeros((100, 4), np.float32), pp)


def test_zbuffer_scratch_left_empty():
    c = configs.room_case(noise=True)
    zb = up.empty_zbuf(c.sweep.pixels, "cuda")
    up.project(dev(c.scan), c.sweep, zbuf=zb)
    up.project(dev(c.scan), c.sweep, zbuf=zb)
    assert bool((zb == -1).all())


# ----------------------------------------------------------------------------- a2


def _normals_compare(pix, depth, pp, precision=up.F32):
    """Per-pixel bound.  The FP32 neighbour vectors a, b are exact or within one rounding, and
    FP32 evaluation of a x b perturbs it by a few 1e-7 |a||b|, so the normal's angle error is
    about 1e-7 / sin(a, b) (sin from the oracle).  Bound used: 1e-6 / sin + 1e-6 rad; FP16
    storage adds up to 2^-11 per component (bound + 2e-3 rad)."""
    n_ref, v_ref, sab = oracle.normals(pix, depth, pp, with_conditioning=True)
    got = host(up.normals(dev(pix), dev(depth), pp, up.Params(), precision)).astype(np.float64)
    v = got[..., 3] != 0
    both = v & v_ref
    ang = angle_between(got[..., :3][both], n_ref[both])
    bound = 1e-6 / sab[both] + 1e-6 + (2e-3 if precision == up.F16 else 0.0)
    assert np.all(ang <= bound), (ang - bound).max()
    # validity differs only at min_cross / orientation near-ties
    diff = v != v_ref
    assert diff.sum() <= max(2, 1e-3 * v_ref.sum()), diff.sum()
    return both.sum()


def test_normals_sweep_parity():
    for cfg in ("room", "tunnel"):
        if cfg == "room":
            c = configs.room_case(noise=True)
            sc, pp = c.scan, c.sweep
        else:
            seq = configs.tunnel_sequence(n_scans=2)
            sc, pp = seq.scan(1), seq.sweep
        depth, idx = oracle.project(sc, pp)
        pix = oracle.pixel_points(sc, idx)
        assert _normals_compare(pix, depth, pp) > 0.8 * (idx >= 0).sum()


def test_normals_fp16_storage():
    c = configs.room_case(noise=True)
    depth, idx = oracle.project(c.scan, c.sweep)
    pix = oracle.pixel_points(c.scan, idx)
    _normals_compare(pix, depth, c.sweep, up.F16)


def test_unproject_matches_table_points():
    pp = synth.keyframe_pano(64, 256)
    rng = np.random.default_rng(22)
    depth = np.where(rng.random((64, 256)) < 0.7, rng.uniform(0.5, 40, (64, 256)), 0).astype(np.float32)
    dirs = up.pano_dirs(pp)
    got = host(up.unproject(dev(depth), pp, dirs))
    ref = oracle.keyframe_points(depth, pp)
    assert np.all((got[..., 3] != 0) == (depth > 0))
    assert np.allclose(got[..., :3], ref[..., :3], rtol=0, atol=2e-6 * depth.max())


# ----------------------------------------------------------------------------- a3


def _kf_buffers(kd, kn4, pp, precision=up.F32):
    kf = up.KeyframeBuffer(pp, "cuda", precision)
    nw = kn4.copy()
    nw[..., 3] = (kd > 0).astype(np.float32)
    kf.set(dev(kd), dev(nw).to(kf.nw.dtype))
    return kf


def _sweep_buffers(sp4, sn4, pp, precision=up.F32):
    sw = up.SweepFrame(pp, "cuda", precision)
    sw.set(dev(sp4), dev(sn4).to(sw.nrm.dtype))
    return sw


def _upper_to_full(a):
    A = np.zeros((6, 6))
    A[np.triu_indices(6)] = a
    return A + np.triu(A, 1).T


def test_icp_step_normal_equations_parity():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    T0 = synth.perturb(IDENTITY, np.random.default_rng(23), 0.03, 0.02)
    kf = _kf_buffers(kd, kn, c.kf)
    sw = _sweep_buffers(sp4, sn4, c.sweep)
    st_ref = oracle.normal_equations(kd, kn, c.kf, sp4, sn4, c.sweep, T0, prm)
    T_ref, st_ref2 = oracle.icp_step(kd, kn, c.kf, sp4, sn4, c.sweep, T0, prm)
    state = up.IcpState(kf)
    state.pose.copy_(pose_dev(T0))
    p = up.Params(max_iters=10)
    up.icp_step(kf, sw, state, p)
    st = state.read_stats()
    A, A_ref = _upper_to_full(st["A"]), _upper_to_full(st_ref["A"])
    assert np.linalg.norm(A - A_ref) <= 1e-5 * np.linalg.norm(A_ref)
    assert abs(st["inliers"] - st_ref["inliers"]) <= 2
    assert st["valid"] == st_ref["valid"]
    dt, dr = rot_err(pose_host(state.pose), T_ref)
    assert dt < 1e-4 and dr < 1e-5
    assert st["status"] == 0


def test_icp_persistent_matches_oracle_iterations():
    """Workload 1: ten Gauss-Newton steps in one persistent launch vs the oracle's loop."""
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf = _kf_buffers(kd, kn, c.kf)
    sw = _sweep_buffers(sp4, sn4, c.sweep)
    state = up.IcpState(kf)
    p = up.Params(max_iters=10)
    up.icp(kf, sw, state, p)
    st = state.read_stats()
    T_ref, st_ref, it_ref = oracle.icp(kd, kn, c.kf, sp4, sn4, c.sweep, IDENTITY, prm, max_iters=10)
    dt, dr = rot_err(pose_host(state.pose), T_ref)
    assert dt < 1e-4 and dr < 1e-5, (dt, dr)
    assert st["iters"] == it_ref
    # and the registration itself is right: within 1 cm / 0.1 deg of the truth
    et, er = rot_err(pose_host(state.pose), c.T_true)
    assert et < 0.01 and er < math.radians(0.1)


def test_icp_persistent_repeatable_and_step_equivalent():
    """The persistent launch equals the same number of single-step launches, and reruns bit-identically."""
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf = _kf_buffers(kd, kn, c.kf)
    sw = _sweep_buffers(sp4, sn4, c.sweep)
    p = up.Params(max_iters=3, eps_rot=0.0, eps_trans=0.0)
    a = up.IcpState(kf)
    up.icp(kf, sw, a, p)
    b = up.IcpState(kf)
    up.icp(kf, sw, b, p)
    s = up.IcpState(kf)
    for _ in range(3):
        up.icp_step(kf, sw, s, p)
    assert torch.equal(a.pose, b.pose)
    dt, dr = rot_err(pose_host(a.pose), pose_host(s.pose))
    assert dt < 1e-9 and dr < 1e-9


def test_icp_full_size_workload2_parity():
    """512 x 2048 keyframe and a 64 x 1024 sweep from the tunnel: one step in the bench's launch form."""
    seq = configs.tunnel_sequence(n_scans=3)
    prm = oracle.Params(accept_quality=0.1)
    kf_ref = oracle.Keyframe(seq.kf)
    sp0, sn0, _, _ = oracle.sweep_frame(seq.scan(0), seq.sweep, prm)
    oracle.fuse(kf_ref, sp0, sn0, seq.sweep, IDENTITY, prm)
    sp4, sn4, _, _ = oracle.sweep_frame(seq.scan(2), seq.sweep, prm)
    kd, kn = kf_ref.depth_f32(), kf_ref.nrm4_f32()
    T0 = synth.relative(seq.poses[0], seq.poses[1])
    kf = _kf_buffers(kd, kn, seq.kf)
    sw = _sweep_buffers(sp4, sn4, seq.sweep)
    state = up.IcpState(kf)
    state.pose.copy_(pose_dev(T0))
    up.icp(kf, sw, state, up.Params(max_iters=1))
    st = state.read_stats()
    T_ref, st_ref = oracle.icp_step(kd, kn, seq.kf, sp4, sn4, seq.sweep, T0, prm)
    A, A_ref = _upper_to_full(st["A"]), _upper_to_full(st_ref["A"])
    assert np.linalg.norm(A - A_ref) <= 1e-5 * np.linalg.norm(A_ref)
    assert abs(st["inliers"] - st_ref["inliers"]) <= 3
    dt, dr = rot_err(pose_host(state.pose), T_ref)
    assert dt < 1e-4 and dr < 1e-5


def test_icp_degenerate_plane_on_gpu():
    from tests.helpers import analytic_sweep, noise_free, rendered_keyframe
    scene = synth.Scene()
    scene.add(synth.PLANE, 0, 0, 0, 0, 0, 1)
    lid = noise_free(configs.LIDAR_16)
    P = synth.pose(synth.rot_zyx(0.1, 0.35), [0, 0, 1.5])
    _, sp4, sn4, _, _ = analytic_sweep(scene, lid, P)
    kp = synth.keyframe_pano(128, 512, 0.3, 30.0)
    kd, kn = rendered_keyframe(scene, kp, P)
    kf = _kf_buffers(kd, kn, kp)
    sw = _sweep_buffers(sp4, sn4, lid.pano())
    state = up.IcpState(kf)
    up.icp(kf, sw, state, up.Params(max_iters=5))
    st = state.read_stats()
    assert st["status"] == 3 and st["iters"] == 1
    assert np.array_equal(pose_host(state.pose), IDENTITY)


def test_icp_empty_keyframe_is_degenerate():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf = _kf_buffers(np.zeros_like(kd), np.zeros_like(kn), c.kf)
    sw = _sweep_buffers(sp4, sn4, c.sweep)
    state = up.IcpState(kf)
    up.icp(kf, sw, state, up.Params(max_iters=5))
    st = state.read_stats()
    assert st["status"] == 3 and st["inliers"] == 0 and st["valid"] == int((sp4[..., 3] != 0).sum())


# ----------------------------------------------------------------------------- a4


def _fuse_compare(kf_ref_before, sp4, sn4, sw_pp, T, prm, precision=up.F32, dtol=2e-6, ntol=1e-4):
    kd = kf_ref_before.depth_f32()
    kn = kf_ref_before.nrm4_f32()
    kf = up.KeyframeBuffer(kf_ref_before.pp, "cuda", precision)
    kf.set(dev(kd), dev(kn).to(kf.nw.dtype))
    sw = _sweep_buffers(sp4, sn4, sw_pp)
    p = up.Params(fuse_d_max=prm.fuse_d_max, fuse_cos_theta_max=prm.fuse_cos_theta_max, w_max=prm.w_max)
    up.fuse(kf, sw, pose_dev(T), p, None)
    ref = oracle.Keyframe(kf_ref_before.pp, kd.astype(np.float64), kn[..., :3].astype(np.float64),
                          kn[..., 3].astype(np.float64))
    fused, filled = oracle.fuse(ref, sp4, sn4, sw_pp, T, prm)
    gd = host(kf.depth).astype(np.float64)
    gn = host(kf.nw).astype(np.float64)
    gw = gn[..., 3]
    # weights: exact, except at similarity-gate near-ties
    wdiff = gw != ref.w
    assert wdiff.sum() <= max(2, 1e-4 * (ref.w > 0).sum()), wdiff.sum()
    same = ~wdiff & (ref.w > 0) & (np.linalg.norm(ref.nrm, axis=-1) > 0.5)
    assert np.allclose(gd[same], ref.depth[same], rtol=dtol, atol=0)
    assert angle_between(gn[..., :3][same], ref.nrm[same]).max() <= ntol
    return fused, filled


def test_fuse_parity_workload1():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf_ref = oracle.Keyframe(c.kf, kd.astype(np.float64), kn[..., :3].astype(np.float64), (kd > 0).astype(np.float64))
    fused, filled = _fuse_compare(kf_ref, sp4, sn4, c.sweep, c.T_true, prm)
    assert fused > 1000


def test_fuse_hole_fill_and_saturation_workload2():
    """New keyframe from a tunnel sweep (hole fill only), then repeated fusion up to the count cap."""
    seq = configs.tunnel_sequence(n_scans=3)
    prm = oracle.Params()
    sp0, sn0, _, _ = oracle.sweep_frame(seq.scan(0), seq.sweep, prm)
    empty = oracle.Keyframe(seq.kf)
    fused, filled = _fuse_compare(empty, sp0, sn0, seq.sweep, IDENTITY, prm)
    assert fused == 0 and filled > 50000
    kf_ref = oracle.Keyframe(seq.kf)
    oracle.fuse(kf_ref, sp0, sn0, seq.sweep, IDENTITY, prm)
    for _ in range(11):
        oracle.fuse(kf_ref, sp0, sn0, seq.sweep, IDENTITY, prm)
    assert kf_ref.w.max() == 10
    sp2, sn2, _, _ = oracle.sweep_frame(seq.scan(2), seq.sweep, prm)
    _fuse_compare(kf_ref, sp2, sn2, seq.sweep, synth.relative(seq.poses[0], seq.poses[2]), prm)


def test_fuse_gated_by_registration_quality():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf = _kf_buffers(kd, kn, c.kf)
    sw = _sweep_buffers(sp4, sn4, c.sweep)
    state = up.IcpState(kf)
    up.icp(kf, sw, state, up.Params(max_iters=10))
    before = kf.depth.clone()
    up.fuse(kf, sw, state.pose, up.Params(accept_quality=1e9), state.stats)
    assert torch.equal(before, kf.depth) and state.read_stats()["accepted"] == 0
    up.fuse(kf, sw, state.pose, up.Params(accept_quality=0.1), state.stats)
    assert not torch.equal(before, kf.depth) and state.read_stats()["accepted"] == 1
    assert bool((kf.zbuf == -1).all())


# ----------------------------------------------------------------------------- whole path


def test_register_equals_prior_icp_motion_chain():
    """upslam_register (prior + persistent ICP + motion update in one launch) equals the
    separate calls upslam_predict_pose -> upslam_icp -> upslam_update_motion."""
    import ctypes
    from paper_2101_00585_gb300 import _abi
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf = _kf_buffers(kd, kn, c.kf)
    sw = _sweep_buffers(sp4, sn4, c.sweep)
    p = up.Params(max_iters=10)
    rng = np.random.default_rng(31)
    prev0 = synth.perturb(IDENTITY, rng, 0.02, 0.01)
    mot0 = synth.perturb(IDENTITY, rng, 0.02, 0.01)
    L = up.lib()
    s = torch.cuda.current_stream().cuda_stream
    ks, ss, ip = kf.struct(), sw.struct(), p.icp()
    # chain of separate entry points
    a = up.IcpState(kf)
    prev_a, mot_a = pose_dev(prev0), pose_dev(mot0)
    assert L.upslam_predict_pose(ctypes.c_void_p(prev_a.data_ptr()), ctypes.c_void_p(mot_a.data_ptr()),
                                 ctypes.c_void_p(a.pose.data_ptr()), ctypes.c_void_p(s)) == 0
    up.icp(kf, sw, a, p)
    assert L.upslam_update_motion(ctypes.c_void_p(prev_a.data_ptr()), ctypes.c_void_p(a.pose.data_ptr()),
                                  ctypes.c_void_p(mot_a.data_ptr()), ctypes.c_void_p(s)) == 0
    # one launch
    b = up.IcpState(kf)
    prev_b, mot_b = pose_dev(prev0), pose_dev(mot0)
    rc = L.upslam_register(ctypes.byref(ks), ctypes.byref(ss), ctypes.c_void_p(prev_b.data_ptr()),
                           ctypes.c_void_p(mot_b.data_ptr()), ctypes.c_void_p(b.pose.data_ptr()), 2,
                           ctypes.byref(ip), ctypes.c_void_p(b.stats.data_ptr()), ctypes.c_void_p(b.ws.data_ptr()),
                           ctypes.c_size_t(b.ws_bytes), ctypes.c_void_p(s))
    assert rc == _abi.OK
    for x, y in ((a.pose, b.pose), (mot_a, mot_b), (a.pose, prev_b)):
        dt, dr = rot_err(pose_host(x), pose_host(y))
        assert dt < 1e-9 and dr < 1e-9
    assert a.read_stats()["iters"] == b.read_stats()["iters"]


def test_track_equals_register_then_fuse():
    """upslam_track (one launch) equals upslam_register followed by upslam_fuse on the same inputs."""
    seq = configs.tunnel_sequence(n_scans=4)
    scans = [seq.scan(k) for k in range(4)]
    p = up.Params(accept_quality=0.1)
    a = up.Tracker(seq.sweep, seq.kf, p, fused=True)
    b = up.Tracker(seq.sweep, seq.kf, p, fused=False)
    for trk in (a, b):
        trk.new_keyframe(dev(scans[0]))
        for k in range(1, 4):
            trk.track(dev(scans[k]))
    torch.cuda.synchronize()
    dt, dr = rot_err(pose_host(a.state.pose), pose_host(b.state.pose))
    assert dt < 1e-9 and dr < 1e-9
    ra, rb = a.state.read_stats(), b.state.read_stats()
    assert ra["accepted"] == rb["accepted"] == 1 and ra["iters"] == rb["iters"]
    assert torch.equal(a.kf.nw[..., 3], b.kf.nw[..., 3])
    assert torch.allclose(a.kf.depth, b.kf.depth, rtol=1e-6, atol=0)
    assert bool((a.kf.zbuf == -1).all()) and bool((b.kf.zbuf == -1).all())


def test_track_scan_one_launch_equals_separate_launches():
    """upslam_track_scan (projection, normals, prior, ICP, keyframe update in one launch) equals
    upslam_project + upslam_normals + upslam_track on the same inputs, bit for bit."""
    seq = configs.tunnel_sequence(n_scans=6)
    scans = [dev(seq.scan(k)) for k in range(6)]
    p = up.Params(accept_quality=0.1)
    a = up.Tracker(seq.sweep, seq.kf, p, front_fused=True)
    b = up.Tracker(seq.sweep, seq.kf, p, front_fused=False)
    assert a.front_fused and not b.front_fused and a.launches_per_track == 1
    for trk in (a, b):
        trk.new_keyframe(scans[0])
        for k in range(1, 6):
            trk.track(scans[k])
    torch.cuda.synchronize()
    assert torch.equal(a.state.pose, b.state.pose)
    assert torch.equal(a.sw.depth, b.sw.depth) and torch.equal(a.sw.idx, b.sw.idx)
    assert torch.equal(a.sw.pix, b.sw.pix) and torch.equal(a.sw.nrm, b.sw.nrm)
    assert torch.equal(a.kf.depth, b.kf.depth) and torch.equal(a.kf.nw, b.kf.nw)
    assert bool((a.sw.zbuf == -1).all()) and bool((a.kf.zbuf == -1).all())
    ra, rb = a.state.read_stats(), b.state.read_stats()
    assert ra["iters"] == rb["iters"] and ra["accepted"] == rb["accepted"] == 1
    # and the sweep buffers equal the oracle's projection (bit-exact) for the last scan
    d_ref, i_ref = oracle.project(seq.scan(5), seq.sweep)
    assert np.array_equal(host(a.sw.idx), i_ref)
    assert np.array_equal(host(a.sw.depth).view(np.uint32), d_ref.view(np.uint32))


def test_persistent_steps_keep_the_exact_association():
    """Every step of the persistent launch associates afresh at the current pose: step k's record must
    equal the oracle's normal equations at the pose the kernel reached after k - 1 steps (inliers within
    the gate's near-ties, J^T J 1e-5), for the tunnel workload at full size."""
    seq = configs.tunnel_sequence(n_scans=3)
    prm = oracle.Params(accept_quality=0.1)
    kf_ref = oracle.Keyframe(seq.kf)
    sp0, sn0, _, _ = oracle.sweep_frame(seq.scan(0), seq.sweep, prm)
    oracle.fuse(kf_ref, sp0, sn0, seq.sweep, IDENTITY, prm)
    sp4, sn4, _, _ = oracle.sweep_frame(seq.scan(2), seq.sweep, prm)
    kd, kn = kf_ref.depth_f32(), kf_ref.nrm4_f32()
    kf = _kf_buffers(kd, kn, seq.kf)
    sw = _sweep_buffers(sp4, sn4, seq.sweep)
    T0 = synth.perturb(synth.relative(seq.poses[0], seq.poses[2]), np.random.default_rng(29), 0.03, 0.01)
    prev = T0
    for k in range(1, 6):
        state = up.IcpState(kf)
        state.pose.copy_(pose_dev(T0))
        up.icp(kf, sw, state, up.Params(max_iters=k, eps_rot=0.0, eps_trans=0.0))
        st = state.read_stats()
        assert st["iters"] == k
        ref = oracle.normal_equations(kd, kn, seq.kf, sp4, sn4, seq.sweep, prev, prm)
        A, A_ref = _upper_to_full(st["A"]), _upper_to_full(ref["A"])
        assert abs(st["inliers"] - ref["inliers"]) <= 3, (k, st["inliers"], ref["inliers"])
        assert np.linalg.norm(A - A_ref) <= 1e-5 * np.linalg.norm(A_ref), k
        prev = pose_host(state.pose)
