"""FP64 CPU oracle for the UPSLAM per-sweep hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The CUDA library never calls it, and
the two share no code: this package compiles ``upslam_oracle.c`` with gcc and
wraps it with ctypes over numpy arrays.

Every function follows a passage of UPSLAM (arXiv 2101.00585):

=====================  =============================================================
``project``            Sec. III-A: points binned into a panoramic depth image
                       (deterministic z-buffer: smallest (range, index) wins)
``pixel_points``       the z-buffer winner's own xyz at every pixel
``normals``            Sec. III-A: cross product of the vectors to two image
                       neighbours
``atrous``             Sec. III-A: edge-avoiding a-trous smoothing of the normals
``icp_step``           Sec. III-B, Eq. 1 (point-to-plane over projective
                       correspondences filtered by Omega_{d,theta}), squared and
                       solved by Gauss-Newton
``fuse``               Sec. III-C: keyframe pixels projected onto the sweep image,
                       similarity-gated, averaged with a count saturated at 10
``quality``            Sec. III-C: inliers / valid sweep measurements
``grid_score``         Sec. III-C: low-resolution alignment checks of candidate poses
``consistency``        Sec. III-C: mutual consistency of two keyframes (moving objects)
``predict_pose``       Sec. IV-F footnote: zero-velocity / zero-acceleration prior
``update_motion``      Sec. IV-F footnote: the last inter-sweep motion
``track``              the per-sweep chain: prior, process_scan, motion update
=====================  =============================================================

Pins that tie it to the paper and to mathematics rather than to itself live in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, replace

import numpy as np

from .atrous import atrous  # noqa: F401  (Sec. III-A normal smoothing)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "upslam_oracle.c")
_SO = os.path.join(_HERE, "_upslam_oracle.so")
_lib = None

DEGENERATE = 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: IEEE round-to-nearest, no FMA contraction."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               _SRC, "-o", _SO, "-lm"])
    return _SO


class Pano(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("el_top", ctypes.c_float),
                ("s_az", ctypes.c_float), ("s_el", ctypes.c_float), ("r_min", ctypes.c_float),
                ("r_max", ctypes.c_float)]


class NormalParams(ctypes.Structure):
    _fields_ = [("jump_rel", ctypes.c_float), ("jump_abs", ctypes.c_float), ("min_cross", ctypes.c_float)]


class IcpParams(ctypes.Structure):
    _fields_ = [("d_max", ctypes.c_float), ("cos_theta_max", ctypes.c_float), ("max_iters", ctypes.c_int32),
                ("min_inliers", ctypes.c_int32), ("eps_rot", ctypes.c_double), ("eps_trans", ctypes.c_double),
                ("pivot_eps", ctypes.c_double), ("loss", ctypes.c_int32), ("loss_delta", ctypes.c_float)]


class IcpStats(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double * 21), ("b", ctypes.c_double * 6), ("sse", ctypes.c_double),
                ("inliers", ctypes.c_int64), ("valid", ctypes.c_int64), ("status", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("xi", ctypes.c_double * 6)]


class FuseParams(ctypes.Structure):
    _fields_ = [("d_max", ctypes.c_float), ("cos_theta_max", ctypes.c_float), ("w_max", ctypes.c_float)]


_F = ctypes.POINTER(ctypes.c_float)
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # UPSLAM_ORACLE_LIB names another build of upslam_oracle.c: the planted-mistake
    # tests load deliberately broken copies through it to show that the pins fail.
    path = os.environ.get("UPSLAM_ORACLE_LIB") or build()
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    sig = {
        "orc_atan2p": (ctypes.c_float, [ctypes.c_float, ctypes.c_float]),
        "orc_bin": (ctypes.c_int, [ctypes.c_float, ctypes.c_float, ctypes.c_float, P(Pano), _I32, _I32, _F]),
        "orc_xform_f32": (None, [_D, ctypes.c_float, ctypes.c_float, ctypes.c_float, _F, _F, _F]),
        "orc_xform_inv_f32": (None, [_D, ctypes.c_float, ctypes.c_float, ctypes.c_float, _F, _F, _F]),
        "orc_dir_table": (None, [P(Pano), _F, _F]),
        "orc_project": (ctypes.c_int64, [_F, ctypes.c_int32, _D, P(Pano), _F, _I32]),
        "orc_normals": (None, [_F, _F, P(Pano), P(NormalParams), _D, _U8, _D]),
        "orc_se3_exp_left": (None, [_D, _D]),
        "orc_solve6": (ctypes.c_int, [_D, _D, ctypes.c_double, _D]),
        "orc_icp_normal_equations": (None, [_F, _F, P(Pano), _F, _F, P(Pano), _D, P(IcpParams), P(IcpStats)]),
        "orc_icp_step": (ctypes.c_int, [_F, _F, P(Pano), _F, _F, P(Pano), _D, P(IcpParams), P(IcpStats)]),
        "orc_icp_residual": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _F, _F, P(Pano), _F, _F, P(Pano), _D,
                                            P(IcpParams), _D, _D, _I64]),
        "orc_fuse": (ctypes.c_int64, [_D, _D, _D, P(Pano), _F, _F, P(Pano), _D, P(FuseParams), _I64]),
        "orc_consistency_flags": (ctypes.c_int64, [_F, P(Pano), _F, P(Pano), _D, ctypes.c_float, ctypes.c_float,
                                                   _U8]),
        "orc_pose_inv_fixed": (None, [_D, _D]),
        "orc_orthonormalise_rows": (None, [_D]),
        "orc_predict_pose": (None, [_D, _D, _D]),
        "orc_update_motion": (None, [_D, _D, _D]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _f(a):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(_F)


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def pano(p) -> Pano:
    """Oracle panorama struct from any object with the seven panorama fields."""
    return Pano(int(p.rows), int(p.cols), float(np.float32(p.el_top)), float(np.float32(p.s_az)),
                float(np.float32(p.s_el)), float(np.float32(p.r_min)), float(np.float32(p.r_max)))


# ----------------------------------------------------------------------------- parameters (readings)

@dataclass
class Params:
    """Thresholds the paper leaves open; these are this implementation's readings."""
    jump_rel: float = 0.05
    jump_abs: float = 0.1
    min_cross: float = 1e-4
    d_max: float = 0.5
    cos_theta_max: float = float(np.cos(np.radians(30.0)))
    max_iters: int = 15
    min_inliers: int = 6
    eps_rot: float = 1e-6
    eps_trans: float = 1e-6
    pivot_eps: float = 1e-12
    fuse_d_max: float = 0.2
    fuse_cos_theta_max: float = float(np.cos(np.radians(30.0)))
    w_max: float = 10.0
    accept_quality: float = 0.3
    # Eq. 1's |.|: 0 squares the point-to-plane error; 1 minimises it as printed (L1) by IRLS with
    # weights 1 / max(|r|, loss_delta)
    loss: int = 0
    loss_delta: float = 0.01
    # coarse-to-fine Omega gate of a whole registration (``icp``): steps 0 .. coarse_iters - 1 gate with
    # d_max, later steps with d_max_fine; 0 steps gate every step with d_max
    coarse_iters: int = 0
    d_max_fine: float = 0.5
    # a-trous smoothing of the sweep normals (Sec. III-A); 0 levels = off
    atrous_levels: int = 0
    atrous_sigma_n: float = 0.5
    atrous_sigma_x: float = 0.02

    def normal_params(self) -> NormalParams:
        return NormalParams(self.jump_rel, self.jump_abs, self.min_cross)

    def icp_params(self) -> IcpParams:
        return IcpParams(self.d_max, self.cos_theta_max, self.max_iters, self.min_inliers, self.eps_rot,
                         self.eps_trans, self.pivot_eps, self.loss, self.loss_delta)

    def fuse_params(self) -> FuseParams:
        return FuseParams(self.fuse_d_max, self.fuse_cos_theta_max, self.w_max)


# ----------------------------------------------------------------------------- FP32 decisions

def atan2p(y: float, x: float) -> float:
    return float(_load().orc_atan2p(float(y), float(x)))


def bin_point(p, pp):
    """(row, col, range) of an FP32 point in panorama pp, or None."""
    v, u, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    ok = _load().orc_bin(float(np.float32(p[0])), float(np.float32(p[1])), float(np.float32(p[2])),
                         ctypes.byref(pano(pp)), ctypes.byref(v), ctypes.byref(u), ctypes.byref(r))
    return (v.value, u.value, r.value) if ok else None


def dir_table(pp):
    rt = np.empty(2 * pp.rows, np.float32)
    ct = np.empty(2 * pp.cols, np.float32)
    _load().orc_dir_table(ctypes.byref(pano(pp)), _f(rt), _f(ct))
    return rt, ct


# ----------------------------------------------------------------------------- a1..a4

def project(pts4: np.ndarray, pp, T: np.ndarray | None = None):
    """Sec. III-A projection with the deterministic z-buffer -> (depth [H,W] f32, idx [H,W] i32)."""
    pts4 = np.ascontiguousarray(pts4, dtype=np.float32)
    depth = np.empty((pp.rows, pp.cols), np.float32)
    idx = np.empty((pp.rows, pp.cols), np.int32)
    Tp = _d(np.ascontiguousarray(T, dtype=np.float64)) if T is not None else None
    _load().orc_project(_f(pts4), pts4.shape[0], Tp, ctypes.byref(pano(pp)), _f(depth),
                        idx.ctypes.data_as(_I32))
    return depth, idx


def pixel_points(pts4: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """[H,W,4] FP32: the winning point's xyz and 1 where a pixel holds a point, else zeros."""
    out = np.zeros(idx.shape + (4,), np.float32)
    m = idx >= 0
    out[m, :3] = pts4[idx[m], :3]
    out[m, 3] = 1.0
    return out


def keyframe_points(depth: np.ndarray, pp) -> np.ndarray:
    """[H,W,4] FP64 points depth * dir(pixel centre) for a keyframe depth image."""
    v = np.arange(pp.rows) + 0.5
    u = np.arange(pp.cols) + 0.5
    el = np.float64(np.float32(pp.el_top)) - v / np.float64(np.float32(pp.s_el))
    az = np.pi - u / np.float64(np.float32(pp.s_az))
    d = depth.astype(np.float64)
    out = np.zeros((pp.rows, pp.cols, 4))
    out[..., 0] = d * np.cos(el)[:, None] * np.cos(az)[None, :]
    out[..., 1] = d * np.cos(el)[:, None] * np.sin(az)[None, :]
    out[..., 2] = d * np.sin(el)[:, None]
    out[..., 3] = (depth > 0).astype(np.float64)
    return out


def normals(pix_pts: np.ndarray, depth: np.ndarray, pp, prm: Params = Params(), with_conditioning: bool = False):
    """Sec. III-A cross-product normals -> (normals [H,W,3] FP64, valid [H,W] bool[, sin(a, b) [H,W]])."""
    pix = np.ascontiguousarray(pix_pts, dtype=np.float32)
    dep = np.ascontiguousarray(depth, dtype=np.float32)
    nrm = np.empty((pp.rows, pp.cols, 3))
    val = np.empty((pp.rows, pp.cols), np.uint8)
    sab = np.empty((pp.rows, pp.cols))
    _load().orc_normals(_f(pix), _f(dep), ctypes.byref(pano(pp)), ctypes.byref(prm.normal_params()), _d(nrm),
                        val.ctypes.data_as(_U8), _d(sab))
    if with_conditioning:
        return nrm, val.astype(bool), sab
    return nrm, val.astype(bool)


def normals4(nrm: np.ndarray, valid: np.ndarray) -> np.ndarray:
    """Pack FP64 normals and their validity into the FP32 [.., 4] layout the kernels read."""
    out = np.zeros(nrm.shape[:-1] + (4,), np.float32)
    out[..., :3] = np.where(valid[..., None], nrm, 0.0)
    out[..., 3] = valid.astype(np.float32)
    return out


def stats_dict(st: IcpStats) -> dict:
    return {"A": np.array(st.A[:]), "b": np.array(st.b[:]), "sse": st.sse, "inliers": st.inliers,
            "valid": st.valid, "status": st.status, "converged": st.converged, "xi": np.array(st.xi[:])}


def _icp_args(kf_depth, kf_nrm4, sp4, sn4):
    kd = np.ascontiguousarray(kf_depth, np.float32)
    kn = np.ascontiguousarray(kf_nrm4, np.float32)
    sp = np.ascontiguousarray(sp4, np.float32)
    sn = np.ascontiguousarray(sn4, np.float32)
    return kd, kn, sp, sn


def normal_equations(kf_depth, kf_nrm4, kp, sp4, sn4, sw, T, prm: Params = Params()) -> dict:
    """Eq. 1 linearised at T: J^T J (upper triangle), J^T r, sum r^2, inliers, valid."""
    kd, kn, sp, sn = _icp_args(kf_depth, kf_nrm4, sp4, sn4)
    st = IcpStats()
    _load().orc_icp_normal_equations(_f(kd), _f(kn), ctypes.byref(pano(kp)), _f(sp), _f(sn), ctypes.byref(pano(sw)),
                                     _d(np.ascontiguousarray(T, np.float64)), ctypes.byref(prm.icp_params()),
                                     ctypes.byref(st))
    return stats_dict(st)


def icp_step(kf_depth, kf_nrm4, kp, sp4, sn4, sw, T, prm: Params = Params()):
    """One Gauss-Newton step of Eq. 1 (squared) -> (new T, stats)."""
    kd, kn, sp, sn = _icp_args(kf_depth, kf_nrm4, sp4, sn4)
    Tn = np.ascontiguousarray(T, np.float64).copy()
    st = IcpStats()
    _load().orc_icp_step(_f(kd), _f(kn), ctypes.byref(pano(kp)), _f(sp), _f(sn), ctypes.byref(pano(sw)), _d(Tn),
                         ctypes.byref(prm.icp_params()), ctypes.byref(st))
    return Tn, stats_dict(st)


def icp(kf_depth, kf_nrm4, kp, sp4, sn4, sw, T0, prm: Params = Params(), max_iters: int | None = None):
    """Iterate icp_step until convergence, a degenerate system, or max_iters -> (T, last stats, steps).
    With prm.coarse_iters > 0, steps from coarse_iters on gate with d_max_fine instead of d_max."""
    T = np.ascontiguousarray(T0, np.float64).copy()
    iters = 0
    st = None
    fine = replace(prm, d_max=prm.d_max_fine)
    for i in range(prm.max_iters if max_iters is None else max_iters):
        Tn, st = icp_step(kf_depth, kf_nrm4, kp, sp4, sn4, sw, T, fine if 0 < prm.coarse_iters <= i else prm)
        iters += 1
        if st["status"] == DEGENERATE:
            break
        T = Tn
        if st["converged"]:
            break
    return T, st, iters


def residual(v, u, kf_depth, kf_nrm4, kp, sp4, sn4, sw, T, prm: Params = Params()):
    """(inlier, r, J, sweep pixel) of keyframe pixel (v, u)."""
    kd, kn, sp, sn = _icp_args(kf_depth, kf_nrm4, sp4, sn4)
    r = ctypes.c_double()
    J = np.zeros(6)
    j = ctypes.c_int64(-1)
    ok = _load().orc_icp_residual(int(v), int(u), _f(kd), _f(kn), ctypes.byref(pano(kp)), _f(sp), _f(sn),
                                  ctypes.byref(pano(sw)), _d(np.ascontiguousarray(T, np.float64)),
                                  ctypes.byref(prm.icp_params()), ctypes.byref(r), _d(J), ctypes.byref(j))
    return bool(ok), r.value, J, j.value


def grid_score(kf_depth, kf_nrm4, kp, sp4, sn4, sw, poses, stride: int, prm: Params = Params()):
    """Sec. III-C loop closure: a grid of a few hundred candidate poses, each scored by a cheap projective
    check at reduced resolution; the winner is then refined by ICP at full resolution.

    Reading: the check is the ICP association of this oracle (keyframe pixel -> sweep pixel, filter
    Omega) on the keyframe sampled every ``stride`` rows and columns; a candidate's score is its number
    of inliers.  -> (scores int64 [n], best: the first candidate with the largest score)."""
    kd = np.zeros_like(np.asarray(kf_depth, np.float32))
    kd[::stride, ::stride] = np.asarray(kf_depth, np.float32)[::stride, ::stride]
    scores = np.array([normal_equations(kd, kf_nrm4, kp, sp4, sn4, sw, np.asarray(T).reshape(3, 4), prm)["inliers"]
                       for T in poses], dtype=np.int64)
    return scores, int(np.argmax(scores)) if len(scores) else -1


def pose_inv_fixed(T) -> np.ndarray:
    """[R | t]^-1 as [R^T | -R^T t], t' summed in a fixed FP64 order (shared by any bit-exact checker)."""
    out = np.empty(12)
    _load().orc_pose_inv_fixed(_d(np.ascontiguousarray(np.asarray(T, np.float64).reshape(12))), _d(out))
    return out.reshape(3, 4)


def consistency(depth_a, pa, depth_b, pb, T_ab, rel: float = 0.05, abs_m: float = 0.2):
    """Sec. III-C mutual consistency check between keyframes A and B (T_ab: pose of B in A).

    A sample of one keyframe is flagged when the other keyframe's rays through and around it (the
    3 x 3 pixels about the one it bins into) measured surfaces beyond it by more than rel * r + abs:
    the other keyframe saw through the sample, which was a moving object.  Both directions use the
    unmodified depths.  -> (flags_a [Ha, Wa] bool, flags_b [Hb, Wb] bool)."""
    da = np.ascontiguousarray(depth_a, np.float32)
    db = np.ascontiguousarray(depth_b, np.float32)
    fa = np.zeros(da.shape, np.uint8)
    fb = np.zeros(db.shape, np.uint8)
    L = _load()
    Tab = np.ascontiguousarray(np.asarray(T_ab, np.float64).reshape(12))
    Tba = np.ascontiguousarray(pose_inv_fixed(Tab).reshape(12))
    L.orc_consistency_flags(_f(da), ctypes.byref(pano(pa)), _f(db), ctypes.byref(pano(pb)), _d(Tab), float(rel),
                            float(abs_m), fa.ctypes.data_as(_U8))
    L.orc_consistency_flags(_f(db), ctypes.byref(pano(pb)), _f(da), ctypes.byref(pano(pa)), _d(Tba), float(rel),
                            float(abs_m), fb.ctypes.data_as(_U8))
    return fa.astype(bool), fb.astype(bool)


def se3_exp_left(xi, T):
    Tn = np.ascontiguousarray(T, np.float64).copy()
    _load().orc_se3_exp_left(_d(np.ascontiguousarray(xi, np.float64)), _d(Tn))
    return Tn


def solve6(A_up, rhs, pivot_eps: float = 1e-12):
    x = np.zeros(6)
    st = _load().orc_solve6(_d(np.ascontiguousarray(A_up, np.float64)), _d(np.ascontiguousarray(rhs, np.float64)),
                            pivot_eps, _d(x))
    return st, x


class Keyframe:
    """FP64 keyframe state: depth [H,W], normals [H,W,3], sample count [H,W]."""

    def __init__(self, pp, depth=None, nrm=None, w=None):
        self.pp = pp
        H, W = pp.rows, pp.cols
        self.depth = np.zeros((H, W)) if depth is None else np.ascontiguousarray(depth, np.float64).copy()
        self.nrm = np.zeros((H, W, 3)) if nrm is None else np.ascontiguousarray(nrm, np.float64).copy()
        self.w = np.zeros((H, W)) if w is None else np.ascontiguousarray(w, np.float64).copy()

    def depth_f32(self) -> np.ndarray:
        return self.depth.astype(np.float32)

    def nrm4_f32(self) -> np.ndarray:
        out = np.zeros(self.depth.shape + (4,), np.float32)
        out[..., :3] = self.nrm
        out[..., 3] = self.w
        return out


def fuse(kf: Keyframe, sp4, sn4, sw, T, prm: Params = Params()):
    """Sec. III-C keyframe update in place -> (pixels averaged, pixels hole-filled)."""
    sp4 = np.ascontiguousarray(sp4, np.float32).reshape(-1, 4)
    sn4 = np.ascontiguousarray(sn4, np.float32).reshape(-1, 4)
    filled = ctypes.c_int64()
    fused = _load().orc_fuse(_d(kf.depth), _d(kf.nrm), _d(kf.w), ctypes.byref(pano(kf.pp)), _f(sp4), _f(sn4),
                             ctypes.byref(pano(sw)), _d(np.ascontiguousarray(T, np.float64)),
                             ctypes.byref(prm.fuse_params()), ctypes.byref(filled))
    return int(fused), int(filled.value)


def quality(stats: dict) -> float:
    """Sec. III-C registration quality: inliers / valid sweep measurements."""
    return float(stats["inliers"]) / max(1, int(stats["valid"]))


# ----------------------------------------------------------------------------- whole sweep

def sweep_frame(scan4: np.ndarray, sw, prm: Params = Params()):
    """project -> pixel points -> normals (-> a-trous smoothing when prm.atrous_levels > 0) for one sweep:
    (sp4 [H,W,4] f32, sn4 [H,W,4] f32, depth, idx)."""
    depth, idx = project(scan4, sw)
    sp4 = pixel_points(scan4, idx)
    nrm, val = normals(sp4, depth, sw, prm)
    if prm.atrous_levels > 0:
        nrm, val = atrous(sp4, normals4(nrm, val)[..., :3], val, prm.atrous_levels, prm.atrous_sigma_n,
                          prm.atrous_sigma_x)
    return sp4, normals4(nrm, val), depth, idx


def process_scan(kf: Keyframe, scan4, sw, T0, prm: Params = Params()):
    """One whole hot-path step: sweep frame, ICP from T0, fusion when accepted -> (T, stats, iters, accepted)."""
    sp4, sn4, _, _ = sweep_frame(scan4, sw, prm)
    T, st, iters = icp(kf.depth_f32(), kf.nrm4_f32(), kf.pp, sp4, sn4, sw, T0, prm)
    accepted = st is not None and st["status"] != DEGENERATE and quality(st) >= prm.accept_quality
    if accepted:
        fuse(kf, sp4, sn4, sw, T, prm)
    return T, st, iters, accepted


# ----------------------------------------------------------------------------- motion prior

def _pose12(T) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(T, np.float64).reshape(12))


def orthonormalise_rows(T) -> np.ndarray:
    """Gram-Schmidt on the rotation rows of a 3x4 pose (r2 = r0 x r1)."""
    out = _pose12(T).copy()
    _load().orc_orthonormalise_rows(_d(out))
    return out.reshape(3, 4)


def predict_pose(T_prev, M=None) -> np.ndarray:
    """Sec. IV-F footnote: the ICP initial guess.  M None: zero velocity (T_prev); else zero
    acceleration, T_prev M with the rotation re-orthonormalised."""
    out = np.empty(12)
    _load().orc_predict_pose(_d(_pose12(T_prev)), None if M is None else _d(_pose12(M)), _d(out))
    return out.reshape(3, 4)


def update_motion(T_prev, T) -> np.ndarray:
    """Sec. IV-F footnote: the last inter-sweep motion M = T_prev^-1 T, re-orthonormalised."""
    out = np.empty(12)
    _load().orc_update_motion(_d(_pose12(T_prev)), _d(_pose12(T)), _d(out))
    return out.reshape(3, 4)


def track(kf: Keyframe, scan4, sw, T_prev, M, prm: Params = Params(), constant_velocity: bool = True):
    """One sweep of a tracked sequence: the prior from (T_prev, M), process_scan, then the motion
    update.  -> (T, stats, iters, accepted, M_new); the next sweep's T_prev is T."""
    T0 = predict_pose(T_prev, M if constant_velocity else None)
    T, st, iters, accepted = process_scan(kf, scan4, sw, T0, prm)
    return T, st, iters, accepted, update_motion(T_prev, T)
