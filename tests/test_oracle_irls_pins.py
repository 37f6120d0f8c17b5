"""Pins of the absolute-error (L1) reading of Eq. 1, minimised by IRLS in the oracle.

Eq. 1 (Sec. III-B) prints the point-to-plane error inside |.|.  The plain path squares it;
``loss = 1`` minimises the absolute error by iteratively reweighted least squares with
weights 1 / max(|r|, delta).  Pinned by:

* a delta far above every residual makes all weights equal, so the step equals the
  squared-error step (the common factor cancels in A^-1 b);
* the weighted normal equations equal the per-correspondence definition assembled from
  ``oracle.residual`` (a separate entry point of the oracle) pixel by pixel;
* a minority of gross outliers (slabs in front of two walls, present in the sweep only)
  biases the squared-error solution and leaves the absolute-error one near the truth.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle
import synth
from synth import configs
from tests.helpers import IDENTITY, room_sweep_and_keyframe


def _full(a):
    A = np.zeros((6, 6))
    A[np.triu_indices(6)] = a
    return A + np.triu(A, 1).T


def test_large_delta_gives_the_squared_error_step():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    T0 = synth.perturb(IDENTITY, np.random.default_rng(51), 0.03, 0.01)
    l2 = oracle.normal_equations(kd, kn, c.kf, sp4, sn4, c.sweep, T0, prm)
    big = dataclasses.replace(prm, loss=1, loss_delta=1e6)
    l1 = oracle.normal_equations(kd, kn, c.kf, sp4, sn4, c.sweep, T0, big)
    assert l1["inliers"] == l2["inliers"]
    assert np.allclose(l1["A"] * 1e6, l2["A"], rtol=1e-12, atol=0)
    assert np.allclose(l1["b"] * 1e6, l2["b"], rtol=1e-12, atol=1e-18)
    _, s2 = oracle.icp_step(kd, kn, c.kf, sp4, sn4, c.sweep, T0, prm)
    _, s1 = oracle.icp_step(kd, kn, c.kf, sp4, sn4, c.sweep, T0, big)
    assert np.allclose(s1["xi"], s2["xi"], rtol=1e-9, atol=1e-15)


def test_weighted_normal_equations_match_per_pixel_definition():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    T0 = synth.perturb(IDENTITY, np.random.default_rng(52), 0.02, 0.01)
    p1 = dataclasses.replace(prm, loss=1, loss_delta=0.004)
    st = oracle.normal_equations(kd, kn, c.kf, sp4, sn4, c.sweep, T0, p1)
    A = np.zeros((6, 6))
    b = np.zeros(6)
    sse = 0.0
    n = 0
    for v in range(c.kf.rows):
        for u in range(c.kf.cols):
            ok, r, J, _ = oracle.residual(v, u, kd, kn, c.kf, sp4, sn4, c.sweep, T0, prm)
            if not ok:
                continue
            w = 1.0 / max(abs(r), float(np.float32(0.004)))  # delta is passed as FP32
            A += w * np.outer(J, J)
            b += w * J * r
            sse += w * r * r
            n += 1
    assert st["inliers"] == n
    assert np.allclose(_full(st["A"]), A, rtol=1e-10, atol=0)
    assert np.allclose(st["b"], b, rtol=1e-10, atol=1e-12)
    assert abs(st["sse"] - sse) <= 1e-10 * sse


def test_absolute_error_resists_outlier_slabs():
    c = configs.room_case(noise=True)
    scene = synth.Scene(name="room_with_slabs", prims=c.scene.prims.copy())
    scene.add(synth.OBB, 4.75, 0.0, 1.5, 0.05, 1.5, 1.2, 0.0)    # 0.3 m in front of the x = +5 wall
    scene.add(synth.OBB, 0.0, -3.75, 1.5, 1.5, 0.05, 1.2, 0.0)   # 0.3 m in front of the y = -4 wall
    sc = synth.scan(scene, c.lidar, c.P_w_s, np.random.default_rng(53))
    prm = oracle.Params(max_iters=40)
    sp4, sn4, _, _ = oracle.sweep_frame(sc, c.sweep, prm)
    d, _, _ = synth.render_keyframe(c.scene, c.kf, c.P_w_kf)
    kd = d.astype(np.float32)
    kn, kv = oracle.normals(oracle.keyframe_points(kd, c.kf).astype(np.float32), kd, c.kf, prm)
    kn4 = oracle.normals4(kn, kv)
    T2, _, _ = oracle.icp(kd, kn4, c.kf, sp4, sn4, c.sweep, IDENTITY, prm)
    T1, st1, _ = oracle.icp(kd, kn4, c.kf, sp4, sn4, c.sweep, IDENTITY,
                            dataclasses.replace(prm, loss=1, loss_delta=0.01))
    e2 = synth.pose_error(T2, c.T_true)[0]
    e1 = synth.pose_error(T1, c.T_true)[0]
    assert e2 > 0.01, e2          # the slabs do bias the squared error
    assert e1 < 0.5 * e2 and e1 < 0.01, (e1, e2)
