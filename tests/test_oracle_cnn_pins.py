"""Pins of the FP64 pose-proposal network (no GPU).

The network is not in the paper, so the pins come from mathematics: finite differences for every gradient, a
library correlation for the convolution indexing, the adjoint identity of im2col / col2im, and Adam's closed-form
first step.
"""
from __future__ import annotations

import numpy as np
import scipy.signal

from oracle import cnn


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 12, 20, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    y = (cnn.im2col(x) @ w.reshape(4, -1).T).reshape(2, 6, 10, 4)
    for b in range(2):
        for co in range(4):
            ref = np.zeros((12, 20))
            for ci in range(3):
                ref += scipy.signal.correlate2d(np.pad(x[b, :, :, ci], 1), w[co, :, :, ci], mode="valid")
            assert np.allclose(y[b, :, :, co], ref[::2, ::2], atol=1e-12)


def test_col2im_is_the_adjoint_of_im2col():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 8, 12, 5))
    d = rng.standard_normal((2 * 4 * 6, 45))
    assert np.isclose(np.sum(cnn.im2col(x) * d), np.sum(x * cnn.col2im(d, x.shape)), rtol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    p = cnn.init_params(4)
    x = rng.standard_normal((2, cnn.IN_H, cnn.IN_W, 8))
    target = rng.standard_normal((2, 6))
    wts = np.array([4.0, 4.0, 4.0, 1.0, 1.0, 1.0])
    out, cache = cnn.forward(p, x)
    L, dout = cnn.loss(out, target, wts)
    g = cnn.backward(p, cache, dout)
    eps = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        idx = rng.choice(flat.size, size=min(4, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            Lp = cnn.loss(cnn.forward(p, x)[0], target, wts)[0]
            flat[i] = old - eps
            Lm = cnn.loss(cnn.forward(p, x)[0], target, wts)[0]
            flat[i] = old
            fd = (Lp - Lm) / (2 * eps)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-4 * max(1e-3, abs(fd), abs(an)), (name, i, fd, an)


def test_adam_first_step_closed_form():
    p = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.5, -0.25, 1e-3])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    cnn.adam_step(p, g, m, v, 1, lr=0.1)
    # bias-corrected first moments equal g and second moments g^2: the step is lr * g / (|g| + eps)
    want = np.array([1.0, -2.0, 3.0]) - 0.1 * g["a"] / (np.abs(g["a"]) + 1e-8)
    assert np.allclose(p["a"], want, rtol=1e-12)


def test_downsample_means_only_the_pixels_holding_samples():
    """Each cell is the mean of (depth / scale, nx, ny, nz) over its pixels that hold a sample (depth > 0 and a
    normal flagged valid); cells without one are zero."""
    depth = np.zeros((4, 8), np.float32)
    nrm4 = np.zeros((4, 8, 4), np.float32)
    depth[0:2, 0:2] = 6.0  # cell (0, 0): four samples facing +x
    nrm4[0:2, 0:2] = (1, 0, 0, 1)
    depth[0, 2], nrm4[0, 2] = 2.0, (0, 1, 0, 1)  # cell (0, 1): two samples ...
    depth[1, 3], nrm4[1, 3] = 4.0, (0, 0, 1, 1)
    depth[0, 3], nrm4[0, 3] = 100.0, (1, 1, 1, 0)  # ... a depth without a valid normal ...
    nrm4[1, 2] = (1, 0, 0, 1)  # ... and a normal without a depth
    out = cnn.downsample(depth, nrm4, 2, 4, depth_scale=2.0)
    assert np.allclose(out[0, 0], [3.0, 1.0, 0.0, 0.0], atol=0, rtol=1e-15)
    assert np.allclose(out[0, 1], [1.5, 0.0, 0.5, 0.5], atol=0, rtol=1e-15)
    assert not out[1].any() and not out[0, 2:].any()
