"""Pins of the a-trous normal smoothing oracle (Sec. III-A) against mathematics, not against itself.

* with the edge-stopping weights switched off (huge sigmas) one level is a B3-spline
  correlation with holes, which scipy.ndimage computes independently;
* a constant normal field is a fixed point;
* a crease (normal edge) and a depth step (tangent-plane edge) stop the smoothing, and the
  same inputs with the corresponding sigma opened up do smooth across them;
* seeded noise on a plane is reduced;
* rolling the panorama by whole columns commutes with the filter (the azimuth wraps).
"""
import math

import numpy as np
import pytest
from scipy import ndimage

from oracle.atrous import atrous

# the cubic B-spline smoothing kernel of the a-trous transform: the binomial row C(4, k) / 2^4, taken
# from its definition here rather than from the oracle
B3 = np.array([math.comb(4, k) for k in range(5)], np.float64) / 16.0

H, W = 12, 40


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _plane_points(z=0.0):
    """Points on the plane z = const below a sensor at the origin, one per pixel."""
    u = np.arange(W)[None, :] * np.ones((H, 1))
    v = np.arange(H)[:, None] * np.ones((1, W))
    P = np.stack([3.0 + 0.1 * v, 0.05 * u - 1.0, np.full((H, W), z)], axis=-1)
    return P


def _noisy_plane_normals(rng, sigma=0.1):
    n = np.zeros((H, W, 3))
    n[..., 2] = 1.0
    return _unit(n + sigma * rng.standard_normal((H, W, 3)))


def _dilated_kernel(level):
    s = 1 << level
    k1 = np.zeros(4 * s + 1)
    k1[::s] = B3
    return np.outer(k1, k1)


def _scipy_level(N, V, level):
    """One level with unit weights: correlation of the valid normals, columns wrapped, rows zero-padded."""
    k = _dilated_kernel(level)
    r = k.shape[0] // 2
    out = np.zeros_like(N)
    for c in range(3):
        x = np.where(V, N[..., c], 0.0)
        xp = np.pad(x, ((r, r), (0, 0)), mode="constant")
        xp = np.pad(xp, ((0, 0), (r, r)), mode="wrap")
        out[..., c] = ndimage.correlate(xp, k, mode="constant")[r:-r, r:-r]
    return np.where(V[..., None], _unit(np.where(np.linalg.norm(out, axis=-1, keepdims=True) > 0, out, 1.0)), 0.0)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_unit_weights_equal_scipy_correlation(levels):
    rng = np.random.default_rng(11)
    N = _unit(rng.standard_normal((H, W, 3)) + np.array([0.0, 0.0, 3.0]))
    V = rng.random((H, W)) > 0.2
    P = _plane_points()
    got, gv = atrous(P, N, V, levels=levels, sigma_n=1e9, sigma_x=1e9)
    ref = np.where(V[..., None], N, 0.0)
    for lev in range(levels):
        ref = _scipy_level(ref, V, lev)
    assert np.array_equal(gv, V)
    assert np.abs(got - ref).max() < 1e-12


def test_constant_field_is_fixed_point():
    N = np.zeros((H, W, 3))
    N[..., :] = _unit(np.array([0.2, -0.3, 0.9]))
    V = np.ones((H, W), bool)
    V[3, 5] = False
    got, _ = atrous(_plane_points(), N, V, levels=3)
    assert np.abs(got[V] - N[V]).max() < 1e-15
    assert not got[3, 5].any()


def test_crease_stops_smoothing():
    n1, n2 = np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    N = np.zeros((H, W, 3))
    N[:, : W // 2] = n1
    N[:, W // 2:] = n2
    V = np.ones((H, W), bool)
    P = np.broadcast_to(np.array([5.0, 0.0, 0.0]), (H, W, 3)).copy()  # tangent-plane term inactive
    got, _ = atrous(P, N, V, levels=3, sigma_n=0.3)
    left = got[:, 4: W // 2]
    assert np.degrees(np.arccos(np.clip(left @ n1, -1, 1))).max() < 1e-6
    opened, _ = atrous(P, N, V, levels=3, sigma_n=100.0)
    assert np.degrees(np.arccos(np.clip(opened[:, W // 2 - 1] @ n1, -1, 1))).min() > 1.0


def test_depth_step_stops_smoothing():
    rng = np.random.default_rng(12)
    N = _noisy_plane_normals(rng, 0.05)
    P = _plane_points()
    P[:, W // 2:, 2] = 1.0  # a 1 m step along the normal
    V = np.ones((H, W), bool)
    Vl = V.copy()
    Vl[:, W // 2:] = False  # the left plane alone
    both, _ = atrous(P, N, V, levels=2, sigma_x=0.02)
    alone, _ = atrous(P, N, Vl, levels=2, sigma_x=0.02)
    cols = slice(4, W // 2)
    assert np.abs(both[:, cols] - alone[:, cols]).max() < 1e-9
    opened, _ = atrous(P, N, V, levels=2, sigma_x=1e6)
    assert np.abs(opened[:, W // 2 - 2: W // 2] - alone[:, W // 2 - 2: W // 2]).max() > 1e-3


def test_noise_is_reduced():
    rng = np.random.default_rng(13)
    N = _noisy_plane_normals(rng, 0.1)
    V = np.ones((H, W), bool)
    got, _ = atrous(_plane_points(), N, V, levels=3)
    err_in = np.degrees(np.arccos(np.clip(N[..., 2], -1, 1))).mean()
    err_out = np.degrees(np.arccos(np.clip(got[..., 2], -1, 1))).mean()
    assert err_out < err_in / 3.0


def test_column_roll_commutes():
    rng = np.random.default_rng(14)
    N = _noisy_plane_normals(rng, 0.2)
    P = _plane_points() + 0.01 * rng.standard_normal((H, W, 3))
    V = rng.random((H, W)) > 0.1
    a, _ = atrous(P, N, V, levels=3)
    k = 7
    b, _ = atrous(np.roll(P, k, 1), np.roll(N, k, 1), np.roll(V, k, 1), levels=3)
    assert np.abs(np.roll(a, k, 1) - b).max() < 1e-15


def test_isolated_pixel_keeps_its_normal():
    N = np.zeros((H, W, 3))
    V = np.zeros((H, W), bool)
    N[6, 10] = _unit(np.array([1.0, 2.0, 2.0]))
    V[6, 10] = True
    got, gv = atrous(_plane_points(), N, V, levels=3)
    assert np.array_equal(gv, V)
    assert np.abs(got[6, 10] - N[6, 10]).max() < 1e-15
