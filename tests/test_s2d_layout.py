"""The pose network's first layer runs as a 2x2 space-to-depth convolution.

The library's GEMM for the 3x3 stride-2 pad-1 convolution over the 8-channel input reads the input as
32-channel pixels (Y, X) = input pixels (2Y + dy, 2X + dx), channel 16 dy + 8 dx + c, and applies four
taps (ty, tx) at (oy + ty - 1, ox + tx - 1) with weights placed by ``s2d_feature_source``.  These tests
check that reformulation on the CPU against the plain convolution, written out from its definition.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2101_00585_gb300.proposal import S2D_FEATURES, s2d_feature_source


def _conv3x3_s2(x, w):
    """Plain 3x3 stride-2 pad-1 convolution: x [H][W][C], w [N][3][3][C] -> [H/2][W/2][N]."""
    H, W, C = x.shape
    out = np.zeros((H // 2, W // 2, w.shape[0]))
    for oy in range(H // 2):
        for ox in range(W // 2):
            for ky in range(3):
                for kx in range(3):
                    y, xx = 2 * oy + ky - 1, 2 * ox + kx - 1
                    if 0 <= y < H and 0 <= xx < W:
                        out[oy, ox] += w[:, ky, kx, :] @ x[y, xx]
    return out


def _conv_s2d(x, w):
    """The same through the space-to-depth form with the library's feature order."""
    H, W, C = x.shape
    xs = np.zeros((H // 2, W // 2, 32))
    for dy in range(2):
        for dx in range(2):
            xs[:, :, 16 * dy + 8 * dx:16 * dy + 8 * dx + 8] = x[dy::2, dx::2]
    w72 = w.reshape(w.shape[0], 72)
    w2 = np.zeros((w.shape[0], S2D_FEATURES))
    for f in range(S2D_FEATURES):
        src = s2d_feature_source(f)
        if src >= 0:
            w2[:, f] = w72[:, src]
    out = np.zeros((H // 2, W // 2, w.shape[0]))
    for oy in range(H // 2):
        for ox in range(W // 2):
            cols = np.zeros(S2D_FEATURES)
            for tap in range(4):
                Y, X = oy + (tap >> 1) - 1, ox + (tap & 1) - 1
                if 0 <= Y < H // 2 and 0 <= X < W // 2:
                    cols[32 * tap:32 * tap + 32] = xs[Y, X]
            out[oy, ox] = w2 @ cols
    return out


def test_feature_order_covers_every_3x3_weight_once():
    src = [s2d_feature_source(f) for f in range(S2D_FEATURES)]
    used = [s for s in src if s >= 0]
    assert sorted(used) == list(range(72))
    # the first 16 features (tap (0, 0), dy = 0) are unused: the weight gradient's feature of ones goes there
    assert all(s < 0 for s in src[:16])


@pytest.mark.parametrize("shape", [(8, 12), (4, 4), (6, 2)])
def test_space_to_depth_equals_the_3x3_stride2_convolution(shape):
    rng = np.random.default_rng(sum(shape))
    H, W = shape
    x = rng.standard_normal((H, W, 8))
    w = rng.standard_normal((5, 3, 3, 8))
    assert np.allclose(_conv_s2d(x, w), _conv3x3_s2(x, w), rtol=0, atol=1e-12)
