"""FP64 reference of the edge-avoiding a-trous normal smoothing (TEST INFRASTRUCTURE ONLY).

Per UPSLAM Sec. III-A, normals built from cross products of neighbouring pixels carry a lot of
noise, so they are smoothed by a filter that stops at edges: the a-trous wavelet filter of
Dammertz et al. (2010).  Per Sec. III-B, a little too much smoothing of the sweep normals is
harmless and even helps ICP converge.  The paper gives no filter parameters.  The reading used here, restated from the
published method and not from any code:

* Level l = 0 .. levels-1 convolves with the separable B3-spline taps [1, 4, 6, 4, 1] / 16
  on a 5 x 5 grid whose holes grow with the level: taps sit 2^l pixels apart.  Columns wrap
  (a full panorama turn); rows beyond the image are skipped.
* Each tap is scaled by an edge-stopping weight
      w(p, q) = exp(-|N_p - N_q|^2 / sigma_n^2) * exp(-(N_p . (P_q - P_p))^2 / (sigma_x |P_p|)^2):
  the normal difference stops smoothing across creases; the distance of q from p's tangent
  plane, relative to p's range, stops it across depth edges and keeps it along oblique
  planes.
* Only valid pixels (a normal was computed) take part.  A valid pixel becomes the
  normalised weighted sum of its valid taps (the centre tap always counts, with weight
  36/256); invalid pixels stay invalid.
"""
from __future__ import annotations

import numpy as np

TAPS = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 16.0


def _neighbour(A: np.ndarray, dr: int, dc: int, fill) -> np.ndarray:
    """out[v, u] = A[v + dr, (u + dc) mod W], or fill where v + dr is outside [0, H)."""
    H = A.shape[0]
    out = np.full_like(A, fill)
    rolled = np.roll(A, -dc, axis=1)
    if dr >= 0:
        if dr < H:
            out[:H - dr] = rolled[dr:]
    else:
        if -dr < H:
            out[-dr:] = rolled[:H + dr]
    return out


def atrous(pix_pts: np.ndarray, nrm: np.ndarray, valid: np.ndarray, levels: int = 3, sigma_n: float = 0.5,
           sigma_x: float = 0.02):
    """Smooth a normal image.

    pix_pts [H, W, >=3] points of the pixels (sweep: the z-buffer winners), nrm [H, W, 3],
    valid [H, W] bool.  -> (smoothed normals [H, W, 3] FP64, valid [H, W] bool).
    """
    P = np.asarray(pix_pts, np.float64)[..., :3]
    V = np.asarray(valid, bool)
    N = np.where(V[..., None], np.asarray(nrm, np.float64)[..., :3], 0.0)
    rng = np.linalg.norm(P, axis=-1)
    inv_sn2 = 1.0 / (sigma_n * sigma_n)
    scale2 = np.where(V, (sigma_x * rng) ** 2, 1.0)
    for lev in range(levels):
        s = 1 << lev
        acc = np.zeros_like(N)
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                h = TAPS[dy + 2] * TAPS[dx + 2]
                Nq = _neighbour(N, s * dy, s * dx, 0.0)
                Pq = _neighbour(P, s * dy, s * dx, 0.0)
                Vq = _neighbour(V, s * dy, s * dx, False)
                dn2 = np.sum((N - Nq) ** 2, axis=-1)
                dpl = np.sum(N * (Pq - P), axis=-1)
                w = h * np.exp(-dn2 * inv_sn2) * np.exp(-(dpl * dpl) / scale2)
                w = np.where(V & Vq, w, 0.0)
                acc += w[..., None] * Nq
        norm = np.linalg.norm(acc, axis=-1)
        N = np.where(V[..., None], acc / np.where(norm > 0, norm, 1.0)[..., None], 0.0)
    return N, V
