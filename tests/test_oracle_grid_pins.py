"""Pins of the loop-closure grid search oracle (Sec. III-C: a few hundred candidate poses, each scored by
a cheap projective check at reduced resolution; the winner is refined by ICP at full resolution).

* On an exact room (noise-free sweep, rendered keyframe) the true pose wins a grid of candidates
  around it, and candidates a metre or more away score far lower;
* the score does not depend on the order of the candidates;
* the sampled keyframe is a real subsample: with stride 1 the score is the full ICP inlier count,
  and with stride s it is the count over the pixels (s i, s j) alone.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

import oracle
import synth
from synth import configs
from tests.helpers import IDENTITY, analytic_sweep, rendered_keyframe


def _grid(center, steps_xy=(-0.2, 0.0, 0.2), yaws_deg=(-4.0, 0.0, 4.0)):
    out = []
    for dx in steps_xy:
        for dy in steps_xy:
            for yaw in yaws_deg:
                d = synth.pose(synth.rot_zyx(math.radians(yaw)), [dx, dy, 0.0])
                out.append(synth.pose_mul(d, center))
    return out


def _exact_room():
    c = configs.room_case(noise=False)
    _, sp4, sn4, _, _ = analytic_sweep(c.scene, c.lidar, c.P_w_s)
    kd, kn = rendered_keyframe(c.scene, c.kf, c.P_w_kf)
    return c, sp4, sn4, kd, kn


def test_truth_wins_the_grid():
    c, sp4, sn4, kd, kn = _exact_room()
    prm = oracle.Params(d_max=0.1)
    cands = _grid(c.T_true)
    truth = len(cands) // 2  # offsets (0, 0, 0)
    assert np.allclose(cands[truth], c.T_true)
    scores, best = oracle.grid_score(kd, kn, c.kf, sp4, sn4, c.sweep, cands, 2, prm)
    assert best == truth
    assert scores[truth] > 1.2 * np.sort(scores)[-2]
    far = [synth.pose_mul(synth.pose(np.eye(3), [1.5, -1.0, 0.0]), c.T_true)]
    far_scores, _ = oracle.grid_score(kd, kn, c.kf, sp4, sn4, c.sweep, far, 2, prm)
    assert far_scores[0] < 0.3 * scores[truth]


def test_order_free():
    c, sp4, sn4, kd, kn = _exact_room()
    prm = oracle.Params(d_max=0.1)
    cands = _grid(synth.perturb(c.T_true, np.random.default_rng(71), 0.05, 0.02))
    perm = np.random.default_rng(72).permutation(len(cands))
    s1, b1 = oracle.grid_score(kd, kn, c.kf, sp4, sn4, c.sweep, cands, 3, prm)
    s2, b2 = oracle.grid_score(kd, kn, c.kf, sp4, sn4, c.sweep, [cands[i] for i in perm], 3, prm)
    assert np.array_equal(s1[perm], s2)
    assert np.allclose(cands[b1], cands[perm[b2]]) and s1[b1] == s2[b2]


def test_stride_is_a_subsample():
    c, sp4, sn4, kd, kn = _exact_room()
    prm = oracle.Params(d_max=0.1)
    T = synth.perturb(c.T_true, np.random.default_rng(73), 0.03, 0.01)
    s1, _ = oracle.grid_score(kd, kn, c.kf, sp4, sn4, c.sweep, [T], 1, prm)
    assert s1[0] == oracle.normal_equations(kd, kn, c.kf, sp4, sn4, c.sweep, T, prm)["inliers"]
    # stride 4: the inliers of the full set that sit on rows and columns divisible by 4
    hits = 0
    for v in range(0, c.kf.rows, 4):
        for u in range(0, c.kf.cols, 4):
            ok, _, _, _ = oracle.residual(v, u, kd, kn, c.kf, sp4, sn4, c.sweep, T, prm)
            hits += int(ok)
    s4, _ = oracle.grid_score(kd, kn, c.kf, sp4, sn4, c.sweep, [T], 4, prm)
    assert s4[0] == hits


def test_ties_go_to_the_first_candidate():
    """Grid reading: the first candidate with the largest score wins, so equal candidates resolve to the
    earliest one."""
    c, sp4, sn4, kd, kn = _exact_room()
    prm = oracle.Params(d_max=0.1)
    far = synth.pose_mul(synth.pose(np.eye(3), [1.5, -1.0, 0.0]), c.T_true)
    scores, best = oracle.grid_score(kd, kn, c.kf, sp4, sn4, c.sweep, [far, c.T_true, c.T_true, far], 2, prm)
    assert scores[1] == scores[2] > scores[0] == scores[3]
    assert best == 1
