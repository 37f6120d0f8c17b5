"""Pins of the FP64 oracle to the paper and to mathematics (no GPU).

Each test checks the oracle against something other than itself: FP64 library
functions, brute force on tiny inputs, closed forms, invariants, and synthetic
scenes whose exact geometry the ray caster knows.  The paper prints no worked
example, so there are no golden values from it; ``tests/golden/`` holds the
measurement sequence for the closed-form fusion check of Sec. III-C.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from synth import configs
from tests.helpers import (IDENTITY, analytic_sweep, empty_room, noise_free, rendered_keyframe, room_sweep_and_keyframe,
                           tiny_pano)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- a1: binning


def test_atan2p_error_bound():
    """The FP32 atan2 stays within 1e-6 rad of FP64 atan2 over every octant and the axes."""
    rng = np.random.default_rng(1)
    pts = rng.standard_normal((20000, 2)).astype(np.float32)
    special = np.array([[0, 1], [1, 0], [0, -1], [-1, 0], [1, 1], [-1, 1], [1, -1], [-1, -1], [1e-30, 1], [1, 1e-30],
                        [3, -1e-20], [-1e-20, -3]], np.float32)
    pts = np.vstack([pts, special])
    worst = 0.0
    for y, x in pts:
        a = oracle.atan2p(y, x)
        worst = max(worst, abs(a - math.atan2(float(y), float(x))))
    assert worst <= 1e-6
    assert oracle.atan2p(0.0, 0.0) == 0.0
    # -0 counts as +0: the negative x axis maps to +pi, not -pi
    assert oracle.atan2p(-0.0, -1.0) == pytest.approx(math.pi, abs=1e-6)


def _bins_by_bounds(az, el, pp):
    """Brute force: scan every pixel's FP64 angular bounds for the one that holds (az, el)."""
    hits = []
    for v in range(pp.rows):
        top = float(pp.el_top) - v / float(pp.s_el)
        bot = float(pp.el_top) - (v + 1) / float(pp.s_el)
        if not (bot < el <= top):
            continue
        for u in range(pp.cols):
            a_hi = math.pi - u / float(pp.s_az)
            a_lo = math.pi - (u + 1) / float(pp.s_az)
            if a_lo < az <= a_hi or (u == 0 and az == -math.pi):
                hits.append((v, u))
    return hits


@pytest.mark.parametrize("shape", [(4, 8), (8, 16)])
def test_bins_match_brute_force(shape):
    """Each FP32 bin equals the pixel whose FP64 angular bounds contain the point,
    except within 2e-6 rad of a pixel edge (FP32 rounding of the angles)."""
    pp = tiny_pano(*shape)
    rng = np.random.default_rng(2)
    near_edge = 0
    for _ in range(3000):
        p = rng.standard_normal(3).astype(np.float32) * np.float32(5.0)
        got = oracle.bin_point(p, pp)
        x, y, z = (float(c) for c in p)
        az, el = math.atan2(y, x), math.atan2(z, math.hypot(x, y))
        r = math.sqrt(x * x + y * y + z * z)
        edge_el = min(abs(((float(pp.el_top) - el) * float(pp.s_el)) - round((float(pp.el_top) - el) * float(pp.s_el))),
                      1.0) / float(pp.s_el)
        edge_az = min(abs(((math.pi - az) * float(pp.s_az)) - round((math.pi - az) * float(pp.s_az))), 1.0) / float(pp.s_az)
        if min(edge_el, edge_az) < 2e-6:
            near_edge += 1
            continue
        want = _bins_by_bounds(az, el, pp) if float(pp.r_min) <= r <= float(pp.r_max) else []
        if not want:
            assert got is None
        else:
            assert got is not None and (got[0], got[1]) == want[0]
    assert near_edge < 30


def test_round_trip_pixel_centres():
    """project(unproject(v, u, d)) = (v, u) at every pixel centre, and the binned range is d."""
    for pp in (tiny_pano(8, 16), synth.keyframe_pano(64, 256), configs.LIDAR_64.pano()):
        dirs = pp.pixel_dirs()
        rng = np.random.default_rng(3)
        for v in range(0, pp.rows, max(1, pp.rows // 16)):
            for u in range(0, pp.cols, max(1, pp.cols // 64)):
                d = float(rng.uniform(1.0, 50.0))
                p = (dirs[v, u] * d).astype(np.float32)
                got = oracle.bin_point(p, pp)
                assert got is not None and got[:2] == (v, u)
                assert abs(got[2] - d) <= 1e-5 * d


def test_unproject_of_project_within_half_pixel():
    pp = synth.keyframe_pano(128, 512)
    dirs = pp.pixel_dirs()
    rng = np.random.default_rng(4)
    half = 0.5 * max(1 / float(pp.s_az), 1 / float(pp.s_el)) * math.sqrt(2) + 1e-6
    for _ in range(2000):
        p = rng.standard_normal(3)
        p[2] *= 0.3
        p = (p / np.linalg.norm(p) * rng.uniform(1, 40)).astype(np.float32)
        got = oracle.bin_point(p, pp)
        if got is None:
            continue
        d = dirs[got[0], got[1]]
        ang = math.acos(max(-1.0, min(1.0, float(d @ (p / np.linalg.norm(p))))))
        assert ang <= half


def test_zbuffer_is_lexicographic_min_and_order_free():
    """Smallest range wins; equal ranges go to the smaller index; a permutation changes nothing."""
    pp = tiny_pano(8, 16)
    dirs = pp.pixel_dirs()
    rng = np.random.default_rng(5)
    pts, want = [], {}
    for v in range(pp.rows):
        for u in range(pp.cols):
            k = int(rng.integers(0, 4))
            if k == 0:
                continue
            ranges = rng.uniform(1, 10, size=k).astype(np.float32)
            if k >= 2 and rng.random() < 0.5:
                ranges[1] = ranges[0]  # exact tie
            for r in ranges:
                pts.append((v, u, r))
    pts4 = np.zeros((len(pts), 4), np.float32)
    for i, (v, u, r) in enumerate(pts):
        pts4[i, :3] = (dirs[v, u] * float(r)).astype(np.float32)
        pts4[i, 3] = 1
    depth, idx = oracle.project(pts4, pp)
    for i in range(len(pts4)):
        b = oracle.bin_point(pts4[i], pp)
        key = (np.float32(b[2]).view(np.uint32), i)
        k = (b[0], b[1])
        if k not in want or key < want[k]:
            want[k] = key
    for (v, u), (rb, i) in want.items():
        assert idx[v, u] == i
        assert depth[v, u].view(np.uint32) == rb
    assert (idx >= 0).sum() == len(want)
    perm = rng.permutation(len(pts4))
    depth2, idx2 = oracle.project(pts4[perm], pp)
    assert np.array_equal(depth2.view(np.uint32), depth.view(np.uint32))
    # winners are the same points: ties between identical points resolve to the smaller new index
    same = perm[idx2[idx2 >= 0]]
    assert np.all(np.abs(pts4[same] - pts4[idx[idx >= 0]]).max(axis=1) == 0)


# ----------------------------------------------------------------------------- a2: normals


def test_normals_match_analytic_planes():
    """On a noise-free room scan, cross-product normals equal the ray caster's face normals
    wherever the pixel and its neighbours hit the same face."""
    c = configs.room_case(noise=False)
    sc, nrm_s, ids = synth.scan(c.scene, c.lidar, c.P_w_s, None, return_truth=True)
    depth, idx = oracle.project(sc, c.sweep)
    sp4 = oracle.pixel_points(sc, idx)
    n, val = oracle.normals(sp4, depth, c.sweep)
    H, W = idx.shape
    # a face is identified by its primitive and its exact normal (the room's six walls share a primitive)
    face = np.full((H, W), -1, np.int64)
    hit = idx >= 0
    keys = {}
    for v, u in zip(*np.nonzero(hit)):
        i = idx[v, u]
        key = (int(ids[i]),) + tuple(np.round(nrm_s[i], 9))
        face[v, u] = keys.setdefault(key, len(keys))
    checked = 0
    for v in range(1, H - 1):
        for u in range(W):
            nb = [face[v, u], face[v, (u + 1) % W], face[v, u - 1], face[v + 1, u], face[v - 1, u]]
            if face[v, u] < 0 or len(set(nb)) != 1 or not val[v, u]:
                continue
            truth = nrm_s[idx[v, u]]
            # 1e-5 rad: the FP32 coordinates (rounding 2^-24 |P|, about 3e-7 m at 5 m) over neighbour
            # spacings of 0.06 m (azimuth) and 0.17 m (elevation) move the cross product by < 1e-5 rad
            assert math.atan2(float(np.linalg.norm(np.cross(n[v, u], truth))), float(n[v, u] @ truth)) <= 1e-5
            checked += 1
    assert checked > 0.7 * H * W
    # orientation: toward the sensor
    assert np.all((n[val] * sp4[val][:, :3]).sum(-1) < 0)


def test_normal_discontinuity_and_fallback():
    """A depth jump removes a neighbour; the opposite one is used with the sign flipped."""
    pp = tiny_pano(4, 8)
    dirs = pp.pixel_dirs()
    depth = np.full((4, 8), 5.0, np.float32)
    depth[:, 5] = 9.0  # right neighbour of column 4 jumps
    pts = np.zeros((4, 8, 4), np.float32)
    pts[..., :3] = (dirs * depth[..., None]).astype(np.float32)
    pts[..., 3] = 1
    n, val = oracle.normals(pts, depth, pp)
    assert val[1, 4]
    a = pts[1, 4, :3].astype(np.float64) - pts[1, 3, :3]
    b = pts[2, 4, :3].astype(np.float64) - pts[1, 4, :3]
    want = np.cross(a, b)
    want /= np.linalg.norm(want)
    if want @ pts[1, 4, :3] > 0:
        want = -want
    assert np.allclose(n[1, 4], want, atol=1e-12)
    # the last row has no row below: the row above is used
    assert val[3, 2]
    depth[:, 4] = 0
    pts[:, 4] = 0
    n2, val2 = oracle.normals(pts, depth, pp)
    assert not val2[:, 4].any()


def test_normal_discontinuity_threshold_has_both_terms():
    """The neighbour test |r_nb - r| > 0.05 r + 0.1 m (reading of Sec. III-A): at r = 1 m a step of
    0.12 m is within the limit (0.15 m, most of it the absolute term) and a step of 0.17 m is not."""
    pp = tiny_pano(4, 8)
    dirs = pp.pixel_dirs()
    for step, right_usable in ((0.12, True), (0.17, False)):
        depth = np.full((4, 8), 1.0, np.float32)
        depth[:, 5] = np.float32(1.0 + step)
        pts = np.zeros((4, 8, 4), np.float32)
        pts[..., :3] = (dirs * depth[..., None]).astype(np.float32)
        pts[..., 3] = 1
        n, val = oracle.normals(pts, depth, pp)
        assert val[1, 4]
        P = pts[1, 4, :3].astype(np.float64)
        a = pts[1, 5, :3] - P if right_usable else P - pts[1, 3, :3]
        b = pts[2, 4, :3].astype(np.float64) - P
        want = np.cross(a, b)
        want /= np.linalg.norm(want)
        if want @ P > 0:
            want = -want
        assert np.allclose(n[1, 4], want, atol=1e-12), step


# ----------------------------------------------------------------------------- a3: ICP


def test_identity_gives_zero_residual():
    """Exact sweep and exact keyframe of an empty room at the same pose: r = 0, xi = 0."""
    scene = empty_room()
    lid = noise_free(configs.LIDAR_16)
    P = synth.pose(synth.rot_zyx(0.3), [0.5, -0.2, 1.2])
    _, sp4, sn4, _, _ = analytic_sweep(scene, lid, P)
    kp = synth.keyframe_pano(128, 512, 0.3, 30.0)
    kd, kn = rendered_keyframe(scene, kp, P)
    st = oracle.normal_equations(kd, kn, kp, sp4, sn4, lid.pano(), IDENTITY)
    assert st["inliers"] > 5000
    assert math.sqrt(st["sse"] / st["inliers"]) < 1e-6
    T, st2 = oracle.icp_step(kd, kn, kp, sp4, sn4, lid.pano(), IDENTITY)
    assert np.abs(st2["xi"]).max() < 1e-6


def test_known_perturbation_recovered():
    """Workload-1 room, noise-free, 5 cm / 2 deg: Gauss-Newton returns the true pose."""
    c = configs.room_case(noise=False)
    _, sp4, sn4, _, _ = analytic_sweep(c.scene, c.lidar, c.P_w_s)
    kd, kn = rendered_keyframe(c.scene, c.kf, c.P_w_kf)
    T, st, it = oracle.icp(kd, kn, c.kf, sp4, sn4, c.sweep, IDENTITY, oracle.Params(), max_iters=30)
    dt, dr = synth.pose_error(T, c.T_true)
    # 1e-4 m / 1e-5 rad is the parity bound; a noise-free scene leaves only FP32 rounding of the
    # inputs, so the pin is a hundred times tighter
    assert dt < 1e-6 and dr < 1e-7, (dt, dr)
    assert st["converged"] == 1


def test_single_plane_is_degenerate():
    """A lone plane constrains 3 of 6 degrees of freedom: the solve reports DEGENERATE."""
    scene = synth.Scene()
    scene.add(synth.PLANE, 0, 0, 0, 0, 0, 1)
    lid = noise_free(configs.LIDAR_16)
    P = synth.pose(synth.rot_zyx(0.1, 0.35), [0, 0, 1.5])
    _, sp4, sn4, _, _ = analytic_sweep(scene, lid, P)
    kp = synth.keyframe_pano(128, 512, 0.3, 30.0)
    kd, kn = rendered_keyframe(scene, kp, P)
    T, st = oracle.icp_step(kd, kn, kp, sp4, sn4, lid.pano(), IDENTITY)
    assert st["inliers"] > 100
    assert st["status"] == oracle.DEGENERATE
    assert np.array_equal(T, IDENTITY)


def test_jacobian_matches_finite_differences():
    """J = d r / d xi for the left update exp(xi^) T, by central differences."""
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    T = synth.perturb(IDENTITY, np.random.default_rng(9), 0.01, 0.005)
    rng = np.random.default_rng(10)
    done = 0
    eps = 1e-6
    while done < 40:
        v, u = int(rng.integers(0, c.kf.rows)), int(rng.integers(0, c.kf.cols))
        ok, r, J, j = oracle.residual(v, u, kd, kn, c.kf, sp4, sn4, c.sweep, T, prm)
        if not ok:
            continue
        fd = np.zeros(6)
        for a in range(6):
            e = np.zeros(6)
            e[a] = eps
            okp, rp, _, jp = oracle.residual(v, u, kd, kn, c.kf, sp4, sn4, c.sweep, oracle.se3_exp_left(e, T), prm)
            okm, rm, _, jm = oracle.residual(v, u, kd, kn, c.kf, sp4, sn4, c.sweep, oracle.se3_exp_left(-e, T), prm)
            if not (okp and okm and jp == j and jm == j):
                break
            fd[a] = (rp - rm) / (2 * eps)
        else:
            assert np.allclose(fd, J, rtol=1e-5, atol=1e-7)
            done += 1


def test_normal_equations_symmetric_psd():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    st = oracle.normal_equations(kd, kn, c.kf, sp4, sn4, c.sweep, IDENTITY, prm)
    A = np.zeros((6, 6))
    iu = np.triu_indices(6)
    A[iu] = st["A"]
    A = A + np.triu(A, 1).T
    assert np.linalg.eigvalsh(A).min() > 0
    assert st["valid"] == int((sp4[..., 3] != 0).sum())


def test_solve6_matches_lapack():
    rng = np.random.default_rng(11)
    for _ in range(50):
        M = rng.standard_normal((6, 9))
        A = M @ M.T + 1e-3 * np.eye(6)
        rhs = rng.standard_normal(6)
        st, x = oracle.solve6(A[np.triu_indices(6)], rhs)
        assert st == 0
        assert np.allclose(x, np.linalg.solve(A, rhs), rtol=1e-9, atol=1e-12)
    A = np.diag([1.0, 1, 1, 0, 1, 1])
    st, _ = oracle.solve6(A[np.triu_indices(6)], np.ones(6))
    assert st == oracle.DEGENERATE


@pytest.mark.parametrize("scale", [1.0, 1e-3, 1e-9])
def test_se3_exp_matches_matrix_exponential(scale):
    rng = np.random.default_rng(12)
    for _ in range(20):
        xi = rng.standard_normal(6) * scale
        w, v = xi[:3], xi[3:]
        X = np.zeros((4, 4))
        X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
        X[:3, 3] = v
        E = scipy.linalg.expm(X)
        T0 = synth.perturb(IDENTITY, rng, 1.0, 0.7)
        got = oracle.se3_exp_left(xi, T0)
        T04 = np.vstack([T0, [0, 0, 0, 1]])
        assert np.allclose(got, (E @ T04)[:3], atol=1e-12)


def test_association_matches_brute_force():
    """Each keyframe pixel's sweep pixel equals a brute-force search over the sweep
    pixels' FP64 angular bounds (away from pixel edges)."""
    kp = tiny_pano(4, 8, 30.0)
    sw = tiny_pano(6, 12, 25.0)
    rng = np.random.default_rng(13)
    kd = rng.uniform(2.0, 6.0, size=(4, 8)).astype(np.float32)
    kn = np.zeros((4, 8, 4), np.float32)
    kn[..., 0] = -1.0
    kn[..., 3] = 1
    sp4 = np.zeros((6, 12, 4), np.float32)
    sd = sw.pixel_dirs()
    sp4[..., :3] = (sd * 4.0).astype(np.float32)
    sp4[..., 3] = 1
    sn4 = np.zeros_like(sp4)
    sn4[..., 0] = -1.0
    sn4[..., 3] = 1
    T = synth.perturb(IDENTITY, rng, 0.2, 0.1)
    prm = oracle.Params(d_max=1e9, cos_theta_max=-2.0)
    kdirs = kp.pixel_dirs()
    checked = 0
    for v in range(4):
        for u in range(8):
            s = kdirs[v, u] * float(kd[v, u])
            q = T[:, :3].T @ (s - T[:, 3])
            az, el = math.atan2(q[1], q[0]), math.atan2(q[2], math.hypot(q[0], q[1]))
            fe = (float(sw.el_top) - el) * float(sw.s_el)
            fa = (math.pi - az) * float(sw.s_az)
            if min(abs(fe - round(fe)), abs(fa - round(fa))) < 1e-4:
                continue
            want = _bins_by_bounds(az, el, sw)
            ok, r, J, j = oracle.residual(v, u, kd, kn, kp, sp4, sn4, sw, T, prm)
            if not want:
                assert not ok
                continue
            assert ok and j == want[0][0] * sw.cols + want[0][1]
            checked += 1
    assert checked >= 10


# ----------------------------------------------------------------------------- a4: fusion


def _single_ray_setup(meas):
    """Keyframe and sweep of identical 4x8 geometry; one sweep pixel's point at range m along
    the keyframe pixel (1, 3)'s centre ray, facing normal (-1, 0, 0) rotated onto that ray."""
    kp = tiny_pano(4, 8)
    dirs = kp.pixel_dirs()
    d = dirs[1, 3]
    n = -d
    sp4 = np.zeros((4, 8, 4), np.float32)
    sn4 = np.zeros((4, 8, 4), np.float32)
    sp4[1, 3, :3] = (d * meas).astype(np.float32)
    sp4[1, 3, 3] = 1
    sn4[1, 3, :3] = n.astype(np.float32)
    sn4[1, 3, 3] = 1
    return kp, sp4, sn4, n


def test_fusion_closed_form_golden():
    """Sec. III-C: with the count saturated at 10, n <= 10 fusions give the mean of the
    measurements and later ones the recursion d <- (10 d + m) / 11 (golden file)."""
    with open(os.path.join(GOLDEN, "fusion_sequence.json")) as f:
        g = json.load(f)
    kp, _, _, _ = _single_ray_setup(1.0)
    kf = oracle.Keyframe(kp)
    prm = oracle.Params()
    ms = [float(np.float32(m)) for m in g["measurements"]]
    for i, m in enumerate(ms):
        _, sp4, sn4, n = _single_ray_setup(m)
        oracle.fuse(kf, sp4, sn4, kp, IDENTITY, prm)
        n_seen = i + 1
        if n_seen <= 10:
            want_d = sum(ms[:n_seen]) / n_seen
        else:
            k = n_seen - 10
            d10 = sum(ms[:10]) / 10
            want_d = (10 / 11) ** k * d10 + sum((1 / 11) * (10 / 11) ** (k - j) * ms[9 + j] for j in range(1, k + 1))
        assert kf.depth[1, 3] == pytest.approx(want_d, rel=2e-7)
        assert kf.w[1, 3] == min(n_seen, 10)
        assert np.allclose(kf.nrm[1, 3], n, atol=1e-6)
    assert (kf.w > 0).sum() == 1


def test_fusion_constant_measurement_and_gates():
    kp, sp4, sn4, n = _single_ray_setup(5.0)
    kf = oracle.Keyframe(kp)
    prm = oracle.Params()
    for _ in range(15):
        oracle.fuse(kf, sp4, sn4, kp, IDENTITY, prm)
    assert kf.depth[1, 3] == pytest.approx(5.0, rel=1e-6) and kf.w[1, 3] == 10.0
    # a measurement beyond the distance gate leaves the pixel unchanged
    _, sp_far, sn_far, _ = _single_ray_setup(5.0 + 0.3)
    oracle.fuse(kf, sp_far, sn_far, kp, IDENTITY, prm)
    assert kf.depth[1, 3] == pytest.approx(5.0, rel=1e-6) and kf.w[1, 3] == 10.0
    # a normal beyond the angle gate too
    sn_bad = sn4.copy()
    sn_bad[1, 3, :3] = np.cross(n, [0, 0, 1.0]).astype(np.float32) / np.linalg.norm(np.cross(n, [0, 0, 1.0]))
    _, sp_near, _, _ = _single_ray_setup(5.1)
    oracle.fuse(kf, sp_near, sn_bad, kp, IDENTITY, prm)
    assert kf.depth[1, 3] == pytest.approx(5.0, rel=1e-6)


def test_hole_fill_takes_nearest_sample():
    """Empty keyframe pixels take the nearest sweep sample landing on them (w = 1)."""
    kp = tiny_pano(4, 8)
    sw = tiny_pano(8, 16)
    kd = kp.pixel_dirs()
    sp4 = np.zeros((8, 16, 4), np.float32)
    sn4 = np.zeros((8, 16, 4), np.float32)
    # two sweep pixels whose points land on keyframe pixel (2, 5), at ranges 7 and 4
    for (v, u), r in (((4, 10), 7.0), ((5, 11), 4.0)):
        sp4[v, u, :3] = (kd[2, 5] * r).astype(np.float32)
        sp4[v, u, 3] = 1
        sn4[v, u, :3] = (-kd[2, 5]).astype(np.float32)
        sn4[v, u, 3] = 1
    kf = oracle.Keyframe(kp)
    fused, filled = oracle.fuse(kf, sp4, sn4, sw, IDENTITY)
    assert fused == 0 and filled == 1
    assert kf.w[2, 5] == 1.0 and kf.depth[2, 5] == pytest.approx(4.0, rel=1e-6)


def test_sequence_tracks_tunnel():
    """Workload 2 with the oracle: a short stretch of the corridor stays within 3 cm / 0.3 deg."""
    seq = configs.tunnel_sequence(n_scans=12)
    prm = oracle.Params(accept_quality=0.1)
    kf = oracle.Keyframe(seq.kf)
    sp4, sn4, _, _ = oracle.sweep_frame(seq.scan(0), seq.sweep, prm)
    oracle.fuse(kf, sp4, sn4, seq.sweep, IDENTITY, prm)
    T = IDENTITY.copy()
    for k in range(1, 12):
        T, st, it, acc = oracle.process_scan(kf, seq.scan(k), seq.sweep, T, prm)
        assert acc
    dt, dr = synth.pose_error(T, synth.relative(seq.poses[0], seq.poses[11]))
    assert dt < 0.03 and dr < math.radians(0.3)


# ----------------------------------------------------------------------------- thresholds and branches

def test_points_outside_the_range_interval_are_not_binned():
    """a1: a point is binned only when its range lies in [r_min, r_max]."""
    pp = tiny_pano(4, 8, r_min=0.5, r_max=10.0)
    rt, ct = oracle.dir_table(pp)
    el_c, el_s, az_c, az_s = rt[2], rt[3], ct[6], ct[7]  # centre of pixel (1, 3)
    d = np.array([el_c * az_c, el_c * az_s, el_s], np.float64)
    for r, inside in ((0.4, False), (0.6, True), (9.0, True), (11.0, False)):
        got = oracle.bin_point((d * r).astype(np.float32), pp)
        assert (got is not None) == inside, (r, got)
        if inside:
            assert got[:2] == (1, 3)


def test_nearly_collinear_neighbours_give_no_normal():
    """a2 reading: |a x b| < min_cross |a| |b| leaves the pixel without a normal (here 1e-5 < 1e-4)."""
    pts = np.zeros((4, 8, 4), np.float32)
    depth = np.zeros((4, 8), np.float32)
    for (v, u), p in (((1, 1), (2.0, 0.0, 0.0)), ((1, 2), (2.0, 0.1, 0.0)), ((2, 1), (2.0, 0.2, 2e-6))):
        pts[v, u] = (*p, 1.0)
        depth[v, u] = np.linalg.norm(p)
    _, val = oracle.normals(pts, depth, tiny_pano(4, 8))
    assert not val[1, 1]
    pts[2, 1, 2] = 0.1  # b now leaves the line of a: a proper normal
    _, val = oracle.normals(pts, depth, tiny_pano(4, 8))
    assert val[1, 1]


def test_solve6_rejects_a_pivot_below_the_relative_threshold():
    """Degenerate-solve reading: a Cholesky pivot at or below pivot_eps * max diagonal is rank deficiency."""
    iu = np.triu_indices(6)
    st, _ = oracle.solve6(np.diag([1.0, 1.0, 1.0, 1.0, 1.0, 1e-14])[iu], np.ones(6), 1e-12)
    assert st == oracle.DEGENERATE
    st, x = oracle.solve6(np.diag([1.0, 1.0, 1.0, 1.0, 1.0, 1e-10])[iu], np.ones(6), 1e-12)
    assert st == 0 and np.allclose(x, [1, 1, 1, 1, 1, 1e10], rtol=1e-12)


def test_keyframe_pixels_without_a_normal_are_not_correspondences():
    """Eq. 1 pairs keyframe samples (a depth and a normal).  With the normal gate opened (cos = -1), a
    pixel whose normal is missing must still not pair: the normal equations equal those of the same
    keyframe with that pixel's depth removed as well."""
    c, prm, sp4, sn4, kd, kn4 = room_sweep_and_keyframe(noise=False)
    open_gate = oracle.Params(cos_theta_max=-1.0)
    kn_b = kn4.copy()
    kn_b[::3, ::2] = 0.0
    kd_b = kd.copy()
    kd_b[::3, ::2] = 0.0
    a = oracle.normal_equations(kd, kn_b, c.kf, sp4, sn4, c.sweep, c.T_true, open_gate)
    b = oracle.normal_equations(kd_b, kn_b, c.kf, sp4, sn4, c.sweep, c.T_true, open_gate)
    assert a["inliers"] == b["inliers"] > 1000
    assert np.array_equal(a["A"], b["A"]) and np.array_equal(a["b"], b["b"])


def test_convergence_needs_both_rotation_and_translation_small():
    """Convergence reading: a step converges when |omega| < eps_rot and |v| < eps_trans, both.  With one
    threshold made trivial (1 rad or 1 m) and the other unreachable (1e-12), the first step from a 5 cm /
    2 degree offset must not report convergence; with both at their defaults the run converges with
    both norms small."""
    c = configs.room_case(noise=False)
    sp4, sn4, _, _ = oracle.sweep_frame(c.scan, c.sweep, oracle.Params())
    kd, kn4 = rendered_keyframe(c.scene, c.kf, c.P_w_kf)
    for eps_rot, eps_trans in ((1.0, 1e-12), (1e-12, 1.0)):
        prm = oracle.Params(eps_rot=eps_rot, eps_trans=eps_trans)
        _, st = oracle.icp_step(kd, kn4, c.kf, sp4, sn4, c.sweep, IDENTITY, prm)
        xi = np.asarray(st["xi"])
        assert np.linalg.norm(xi[:3]) < 1.0 and np.linalg.norm(xi[3:]) < 1.0
        assert not st["converged"], (eps_rot, eps_trans)
    prm = oracle.Params(max_iters=40)
    _, st, iters = oracle.icp(kd, kn4, c.kf, sp4, sn4, c.sweep, IDENTITY, prm)
    xi = np.asarray(st["xi"])
    assert st["converged"] and iters < 40
    assert np.linalg.norm(xi[:3]) < prm.eps_rot and np.linalg.norm(xi[3:]) < prm.eps_trans


def test_fusion_blends_normals_with_the_sample_count():
    """Sec. III-C with the fusion reading: n <- unit(w n + R m).  Every keyframe normal is n0 with count 2
    and every sweep normal is m (20 degrees apart, inside the gate), at the identity pose: each averaged
    pixel must hold unit(2 n0 + m) with count 3."""
    c = configs.room_case(noise=False)
    prm = oracle.Params()
    sp4, sn4, _, _ = oracle.sweep_frame(c.scan, c.sweep, prm)
    d, _, _ = synth.render_keyframe(c.scene, c.kf, c.P_w_s)  # keyframe at the sweep's own pose
    n0 = np.array([0.0, 0.0, 1.0])
    m = np.array([math.sin(math.radians(20.0)), 0.0, math.cos(math.radians(20.0))])
    sn = sn4.copy()
    sn[sn[..., 3] != 0, :3] = m
    has = d > 0
    kf = oracle.Keyframe(c.kf, d, np.where(has[..., None], n0, 0.0), np.where(has, 2.0, 0.0))
    fused, _ = oracle.fuse(kf, sp4, sn, c.sweep, IDENTITY, prm)
    averaged = kf.w == 3.0
    assert fused == averaged.sum() > 1000
    want = 2.0 * n0 + m.astype(np.float32)  # sweep normals are stored in FP32
    want /= np.linalg.norm(want)
    assert np.abs(kf.nrm[averaged] - want).max() < 1e-12


def test_fusion_measures_depth_in_the_keyframe_frame():
    """Sec. III-C: the averaged-in depth is the sweep sample's range seen from the keyframe, |T P|.  An
    exact sweep from 0.5 m / 10 degrees away, fused with the true pose into an exact keyframe, leaves the
    keyframe depths where the geometry puts them."""
    c = configs.room_case(noise=False, trans_m=0.5, rot_deg=10.0)
    prm = oracle.Params()
    sp4, sn4, _, _ = oracle.sweep_frame(c.scan, c.sweep, prm)
    kd, kn4 = rendered_keyframe(c.scene, c.kf, c.P_w_kf)
    has = kd > 0
    kf = oracle.Keyframe(c.kf, kd.astype(np.float64), kn4[..., :3].astype(np.float64), np.where(has, 1.0, 0.0))
    fused, _ = oracle.fuse(kf, sp4, sn4, c.sweep, c.T_true, prm)
    averaged = kf.w == 2.0
    assert fused == averaged.sum() > 500
    err = np.abs(kf.depth[averaged] - kd[averaged])
    assert np.median(err) < 0.01 and err.max() < 0.1, (np.median(err), err.max())


# ----------------------------------------------------------------------------- motion prior (Sec. IV-F)


def _hat(xi):
    w, v = xi[:3], xi[3:]
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    X[:3, 3] = v
    return X


def _h(T):
    return np.vstack([np.asarray(T).reshape(3, 4), [0, 0, 0, 1]])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_constant_twist_trajectory_is_predicted_exactly(seed):
    """Poses T_k = T_a exp(k xi^) (a constant body twist, built by the matrix exponential): the motion
    from two consecutive poses is exp(xi^) and the zero-acceleration prior gives the next pose."""
    rng = np.random.default_rng(seed)
    Ta = scipy.linalg.expm(_hat(rng.standard_normal(6) * [0.5, 0.5, 0.5, 3, 3, 3]))
    xi = rng.standard_normal(6) * [0.05, 0.05, 0.05, 0.3, 0.3, 0.3]
    traj = [Ta @ scipy.linalg.expm(k * _hat(xi)) for k in range(6)]
    for k in range(1, 5):
        M = oracle.update_motion(traj[k - 1][:3], traj[k][:3])
        assert np.abs(_h(M) - scipy.linalg.expm(_hat(xi))).max() < 1e-12
        T1 = oracle.predict_pose(traj[k][:3], M)
        assert np.abs(T1 - traj[k + 1][:3]).max() < 1e-12, k


def test_zero_velocity_and_identity_motion_return_the_previous_pose():
    rng = np.random.default_rng(3)
    T = scipy.linalg.expm(_hat(rng.standard_normal(6)))[:3]
    assert np.array_equal(oracle.predict_pose(T, None), T)
    # expm's rotation is orthogonal to a few 1e-15, which the re-orthonormalisation removes
    assert np.abs(oracle.predict_pose(T, IDENTITY) - T).max() < 1e-14
    assert np.abs(oracle.update_motion(T, T) - IDENTITY).max() < 1e-14


def test_motion_update_then_prediction_reproduces_the_pose():
    """predict(T_prev, update_motion(T_prev, T)) = T for any two rigid poses."""
    rng = np.random.default_rng(4)
    for _ in range(20):
        A = scipy.linalg.expm(_hat(rng.standard_normal(6) * 2))[:3]
        B = scipy.linalg.expm(_hat(rng.standard_normal(6) * 2))[:3]
        assert np.abs(oracle.predict_pose(A, oracle.update_motion(A, B)) - B).max() < 1e-13


def test_reorthonormalised_rotation_is_orthogonal_and_keeps_the_first_row():
    """A drifted rotation (scaled rows, skewed) comes back on SO(3): R R^T = I to 1e-15, det +1,
    the first row keeps its direction and the second stays in the plane of the first two."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        R = scipy.linalg.expm(_hat(np.r_[rng.standard_normal(3), 0, 0, 0]))[:3, :3]
        D = R * (1 + 1e-3 * rng.standard_normal((3, 1))) + 1e-3 * rng.standard_normal((3, 3))
        T = np.hstack([D, rng.standard_normal((3, 1))])
        out = oracle.orthonormalise_rows(T)
        Q = out[:, :3]
        assert np.abs(Q @ Q.T - np.eye(3)).max() < 1e-15
        assert abs(np.linalg.det(Q) - 1) < 1e-15
        assert np.allclose(out[:, 3], T[:, 3], rtol=0, atol=0)
        assert np.linalg.norm(np.cross(Q[0], D[0])) < 1e-15 * np.linalg.norm(D[0]) * 10
        assert abs(np.dot(Q[1], np.cross(D[0], D[1]))) < 1e-15 * 10
        assert np.dot(Q[1], D[1]) > 0
    # the prior's product is re-orthonormalised
    M = np.hstack([np.eye(3) * (1 + 1e-6), np.zeros((3, 1))])
    P = oracle.predict_pose(IDENTITY, M)
    assert np.abs(P[:, :3] @ P[:, :3].T - np.eye(3)).max() < 1e-15
