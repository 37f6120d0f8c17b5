"""Host-side pieces of the learned proposal (no GPU): the twist labels and the pair motions.

The labels xi = log(D) are checked against the matrix exponential of the twist's 4 x 4 generator
(scipy), independently of the library's SE(3) kernels; the motions against their stated bounds.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
import scipy.linalg

from paper_2101_00585_gb300 import proposal


def _exp(xi):
    """exp of the 4 x 4 generator of xi = (omega, v)."""
    w, v = xi[:3], xi[3:]
    G = np.zeros((4, 4))
    G[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    G[:3, 3] = v
    return scipy.linalg.expm(G)[:3]


@pytest.mark.parametrize("angle", [0.0, 1e-9, 1e-7, 1e-3, 0.5, 2.0, 3.0])
def test_se3_log_inverts_the_exponential(angle):
    rng = np.random.default_rng(int(angle * 1e3) + 7)
    ax = rng.standard_normal(3)
    ax /= np.linalg.norm(ax)
    xi = np.concatenate([ax * angle, rng.uniform(-1.0, 1.0, 3)])
    got = proposal.se3_log(_exp(xi))
    assert np.allclose(got, xi, atol=1e-9, rtol=1e-9), (got, xi)


def test_random_motions_respect_their_bounds():
    rng = np.random.default_rng(5)
    for _ in range(500):
        D = proposal.random_motion(rng, max_t=1.0, max_deg=30.0)
        R, t = D[:, :3], D[:, 3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and math.isclose(np.linalg.det(R), 1.0, abs_tol=1e-12)
        assert np.linalg.norm(t) <= 1.0 + 1e-12
        ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R) - 1.0) / 2.0))))
        assert ang <= 30.0 + 1e-9
        xi = proposal.se3_log(D)
        assert np.allclose(_exp(xi), D, atol=1e-9)
