"""FP64 reference of the pose-proposal network (TEST INFRASTRUCTURE ONLY).

The learned proposal is not part of the paper.  It is a design addition that predicts the initial relative pose
of a keyframe/sweep pair before ICP refines it.  Nothing in the paper pins this network, so its parity is pinned
by mathematics only:
* finite differences for every gradient;
* an independent library correlation for the convolution indexing.

Architecture, NHWC activations, FP64:

    x0 [B, 64, 256, 8]    keyframe (depth, nx, ny, nz) + sweep (depth, nx, ny, nz), downsampled
    4 x (conv 3x3, stride 2, pad 1, bias, ReLU):  8 -> 32 -> 64 -> 128 -> 128 channels
        64x256 -> 32x128 -> 16x64 -> 8x32 -> 4x16
    global average pool -> [B, 128]
    linear 128 -> 6     -> xi_hat = (omega, v), the relative pose keyframe <- sweep

Convolution weights are [C_out, 3, 3, C_in]; the flattened reduction index is (ky * 3 + kx) * C_in + ci.
Loss: mean over the batch of sum_i w_i (xi_hat_i - xi_i)^2.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (8, 32, 64, 128, 128)
IN_H, IN_W = 64, 256


def init_params(seed: int = 0) -> dict:
    """He-normal convolution weights, zero biases, small linear head (FP64)."""
    rng = np.random.default_rng(seed)
    p = {}
    for l in range(4):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        p[f"w{l}"] = rng.standard_normal((co, 3, 3, ci)) * np.sqrt(2.0 / (9 * ci))
        p[f"b{l}"] = np.zeros(co)
    p["wf"] = rng.standard_normal((6, 128)) * np.sqrt(1.0 / 128)
    p["bf"] = np.zeros(6)
    return p


def im2col(x: np.ndarray) -> np.ndarray:
    """[B, H, W, C] -> [B * H/2 * W/2, 9 * C] for a 3x3, stride-2, pad-1 convolution."""
    B, H, W, C = x.shape
    Ho, Wo = H // 2, W // 2
    xp = np.zeros((B, H + 2, W + 2, C))
    xp[:, 1:H + 1, 1:W + 1] = x
    cols = np.empty((B, Ho, Wo, 3, 3, C))
    for ky in range(3):
        for kx in range(3):
            cols[:, :, :, ky, kx, :] = xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :]
    return cols.reshape(B * Ho * Wo, 9 * C)


def col2im(dcols: np.ndarray, shape) -> np.ndarray:
    """Adjoint of im2col: scatter-add [B * Ho * Wo, 9 * C] back to [B, H, W, C]."""
    B, H, W, C = shape
    Ho, Wo = H // 2, W // 2
    d = dcols.reshape(B, Ho, Wo, 3, 3, C)
    dxp = np.zeros((B, H + 2, W + 2, C))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :] += d[:, :, :, ky, kx, :]
    return dxp[:, 1:H + 1, 1:W + 1]


def forward(p: dict, x0: np.ndarray):
    """-> (xi_hat [B, 6], cache)."""
    x = np.asarray(x0, np.float64)
    cache = {"x0": x}
    for l in range(4):
        B, H, W, C = x.shape
        cols = im2col(x)
        co = CHANNELS[l + 1]
        y = cols @ p[f"w{l}"].reshape(co, -1).T + p[f"b{l}"]
        a = np.maximum(y, 0.0).reshape(B, H // 2, W // 2, co)
        cache[f"cols{l}"] = cols
        cache[f"pre{l}"] = y
        cache[f"in{l}"] = x.shape
        x = a
    g = x.mean(axis=(1, 2))
    cache["last"] = x.shape
    cache["g"] = g
    out = g @ p["wf"].T + p["bf"]
    return out, cache


def loss(out: np.ndarray, target: np.ndarray, weights: np.ndarray):
    """-> (loss, d loss / d out)."""
    diff = out - target
    B = out.shape[0]
    L = float(np.sum(weights * diff * diff) / B)
    return L, 2.0 * weights * diff / B


def backward(p: dict, cache: dict, dout: np.ndarray) -> dict:
    """Gradients of every parameter for the given d loss / d out."""
    grads = {"wf": dout.T @ cache["g"], "bf": dout.sum(axis=0)}
    dg = dout @ p["wf"]
    B, H, W, C = cache["last"]
    da = np.broadcast_to(dg[:, None, None, :] / (H * W), (B, H, W, C))
    for l in range(3, -1, -1):
        co = CHANNELS[l + 1]
        dy = da.reshape(-1, co) * (cache[f"pre{l}"] > 0)
        grads[f"w{l}"] = (dy.T @ cache[f"cols{l}"]).reshape(p[f"w{l}"].shape)
        grads[f"b{l}"] = dy.sum(axis=0)
        if l > 0:
            dcols = dy @ p[f"w{l}"].reshape(co, -1)
            da = col2im(dcols, cache[f"in{l}"])
    return grads


def adam_step(p: dict, grads: dict, m: dict, v: dict, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place (Kingma & Ba, bias-corrected)."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * grads[k]
        v[k] = b2 * v[k] + (1 - b2) * grads[k] ** 2
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def downsample(depth: np.ndarray, nrm4: np.ndarray, out_rows: int, out_cols: int, depth_scale: float) -> np.ndarray:
    """Per cell, the mean over pixels holding a sample (depth > 0, flag != 0, nonzero normal) of
    (depth / depth_scale, nx, ny, nz); zeros where none.  -> [out_rows, out_cols, 4]."""
    H, W = depth.shape
    bh, bw = H // out_rows, W // out_cols
    out = np.zeros((out_rows, out_cols, 4))
    for r in range(out_rows):
        for c in range(out_cols):
            d = depth[r * bh:(r + 1) * bh, c * bw:(c + 1) * bw].astype(np.float64)
            n = nrm4[r * bh:(r + 1) * bh, c * bw:(c + 1) * bw].astype(np.float64)
            m = (d > 0) & (n[..., 3] != 0) & (np.abs(n[..., :3]).sum(-1) > 0)
            if m.any():
                out[r, c, 0] = d[m].mean() / depth_scale
                out[r, c, 1:] = n[..., :3][m].mean(axis=0)
    return out


def flatten(p: dict) -> np.ndarray:
    """Parameters in the flat order w0 b0 w1 b1 w2 b2 w3 b3 wf bf."""
    parts = []
    for l in range(4):
        parts += [p[f"w{l}"].ravel(), p[f"b{l}"].ravel()]
    parts += [p["wf"].ravel(), p["bf"].ravel()]
    return np.concatenate(parts)


def unflatten(flat: np.ndarray) -> dict:
    out, o = {}, 0
    for l in range(4):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        out[f"w{l}"] = flat[o:o + co * 9 * ci].reshape(co, 3, 3, ci)
        o += co * 9 * ci
        out[f"b{l}"] = flat[o:o + co]
        o += co
    out["wf"] = flat[o:o + 768].reshape(6, 128)
    o += 768
    out["bf"] = flat[o:o + 6]
    return out
