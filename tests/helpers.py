"""Shared test inputs: seeded synthetic cases built from ``synth`` and the oracle.

Every input here comes from ``synth`` (generation) and ``oracle`` (expected
values); nothing is computed by the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth
from synth import configs

IDENTITY = np.hstack([np.eye(3), np.zeros((3, 1))])


def analytic_sweep(scene, lidar, P_w_s, rng=None):
    """Sweep pixel points and the ray caster's exact normals -> (scan, sp4, sn4, depth, idx)."""
    sc, nrm_s, ids = synth.scan(scene, lidar, P_w_s, rng, return_truth=True)
    sw = lidar.pano()
    depth, idx = oracle.project(sc, sw)
    sp4 = oracle.pixel_points(sc, idx)
    sn4 = np.zeros_like(sp4)
    m = idx >= 0
    sn4[m, :3] = nrm_s[idx[m]].astype(np.float32)
    sn4[m, 3] = 1.0
    return sc, sp4, sn4, depth, idx


def rendered_keyframe(scene, kp, P_w_kf):
    """Exact keyframe: depth along pixel-centre rays and analytic normals -> (depth f32, nrm4 f32)."""
    d, n, _ = synth.render_keyframe(scene, kp, P_w_kf)
    nrm4 = np.zeros(d.shape + (4,), np.float32)
    nrm4[..., :3] = n
    nrm4[..., 3] = (d > 0).astype(np.float32)
    return d.astype(np.float32), nrm4


def empty_room(seed: int = 7):
    s = synth.Scene(name="empty_room")
    s.add(synth.ROOM, -5.0, -4.0, 0.0, 5.0, 4.0, 3.0)
    return s


def noise_free(lidar):
    return synth.Lidar(**{**lidar.__dict__, "sigma": 0.0, "dropout": 0.0})


def tiny_pano(rows, cols, half_fov_deg=30.0, r_min=0.1, r_max=100.0):
    h = math.radians(half_fov_deg)
    return synth.Pano.make(rows, cols, h, -h, r_min, r_max)


def room_sweep_and_keyframe(noise: bool = True):
    """Workload 1 inputs: sweep frame (oracle a1+a2) and keyframe (rendered depth, oracle a2 normals)."""
    c = configs.room_case(noise=noise)
    prm = oracle.Params(max_iters=10)
    sp4, sn4, depth, idx = oracle.sweep_frame(c.scan, c.sweep, prm)
    d, _, _ = synth.render_keyframe(c.scene, c.kf, c.P_w_kf)
    kd = d.astype(np.float32)
    kpts = oracle.keyframe_points(kd, c.kf).astype(np.float32)
    kn, kv = oracle.normals(kpts, kd, c.kf, prm)
    return c, prm, sp4, sn4, kd, oracle.normals4(kn, kv)
