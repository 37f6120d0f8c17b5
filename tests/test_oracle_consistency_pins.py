"""Pins of the keyframe mutual consistency check (Sec. III-C: when switching keyframes, a mutual
consistency check between keyframes filters moving objects from the map).

Reading: a keyframe sample is flagged when the other keyframe's rays through and around it (3 x 3
pixels) measured surfaces beyond it by more than rel * r + abs, i.e. the other keyframe saw
through it.  Pinned by geometry:

* two exact renderings of a static scene from different poses flag (almost) nothing;
* a box present when keyframe A was rendered and gone when B was: A's box samples that B looks
  at are flagged, the room's walls are not, and none of B's samples are (an occluder hides, it is
  not seen through);
* a keyframe checked against itself at the identity flags nothing (every sample re-bins into its
  own pixel at its own range);
* the fixed-order pose inverse is the inverse.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth
from synth import configs
from tests.helpers import IDENTITY


def _room_pair(with_box_in_a: bool):
    c = configs.room_case(noise=False)
    kp = synth.keyframe_pano(256, 1024, 0.3, 30.0)
    P_a = c.P_w_kf
    P_b = synth.pose_mul(P_a, synth.pose(synth.rot_zyx(math.radians(25.0)), [0.8, 0.6, 0.0]))
    scene_a = synth.Scene(name="a", prims=c.scene.prims.copy())
    box = None
    if with_box_in_a:
        # a box standing between the two keyframes and the x = +5 wall
        box = (3.0, 0.2, 1.0, 0.3, 0.3, 1.0)
        scene_a.add(synth.OBB, *box, 0.0)
    da, _, ida = synth.render_keyframe(scene_a, kp, P_a)
    db, _, idb = synth.render_keyframe(c.scene, kp, P_b)
    return kp, da.astype(np.float32), db.astype(np.float32), synth.relative(P_a, P_b), ida, len(c.scene.prims)


def test_static_scene_is_consistent():
    kp, da, db, T_ab, _, _ = _room_pair(False)
    fa, fb = oracle.consistency(da, kp, db, kp, T_ab)
    assert fa.sum() <= 1e-3 * (da > 0).sum(), fa.sum()
    assert fb.sum() <= 1e-3 * (db > 0).sum(), fb.sum()


def test_moving_box_is_removed_from_the_keyframe_that_saw_it():
    kp, da, db, T_ab, ida, n_static = _room_pair(True)
    fa, fb = oracle.consistency(da, kp, db, kp, T_ab)
    on_box = (ida == n_static) & (da > 0)   # the box is the last primitive of scene A
    assert on_box.sum() > 200
    # samples of A on the box that B's panorama covers: B saw the wall behind them
    assert fa[on_box].mean() > 0.9, fa[on_box].mean()
    assert fa[~on_box].sum() <= 1e-3 * (~on_box & (da > 0)).sum()
    assert fb.sum() <= 1e-3 * (db > 0).sum()


def test_identity_flags_nothing():
    kp, da, _, _, _, _ = _room_pair(True)
    fa, fb = oracle.consistency(da, kp, da, kp, IDENTITY)
    assert not fa.any() and not fb.any()


def test_pose_inverse():
    T = synth.perturb(IDENTITY, np.random.default_rng(91), 2.0, 0.8)
    Ti = oracle.pose_inv_fixed(T)
    M = np.vstack([T, [0, 0, 0, 1]])
    assert np.abs(np.vstack([Ti, [0, 0, 0, 1]]) - np.linalg.inv(M)).max() < 1e-14


def _tiny():
    from tests.helpers import tiny_pano
    return tiny_pano(8, 16)


def test_margin_has_relative_and_absolute_parts():
    """At the identity a sample at r = 1 m is seen through only when every depth around it in the other
    keyframe lies beyond r + (0.05 r + 0.2 m) = 1.25 m."""
    pp = _tiny()
    da = np.full((8, 16), 1.0, np.float32)
    for other, flagged in ((1.1, False), (1.2, False), (1.3, True)):
        db = np.full((8, 16), other, np.float32)
        fa, _ = oracle.consistency(da, pp, db, pp, IDENTITY, rel=0.05, abs_m=0.2)
        assert fa.all() if flagged else not fa.any(), other


def test_neighbourhood_covers_the_rows_above_and_below():
    """A sample stays when any depth-holding pixel of the other keyframe's 3 x 3 neighbourhood around it
    lies within the margin, even though the centre pixel saw through it."""
    pp = _tiny()
    da = np.zeros((8, 16), np.float32)
    da[4, 8] = 1.0
    db = np.full((8, 16), 5.0, np.float32)
    fa, _ = oracle.consistency(da, pp, db, pp, IDENTITY)
    assert fa[4, 8]
    for dv, du in ((-1, 0), (1, 0), (-1, -1), (1, 1), (0, 1), (0, -1)):
        db2 = db.copy()
        db2[4 + dv, 8 + du] = 1.0
        fa2, _ = oracle.consistency(da, pp, db2, pp, IDENTITY)
        assert not fa2[4, 8], (dv, du)
