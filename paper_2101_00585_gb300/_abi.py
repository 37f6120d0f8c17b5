"""ctypes view of the C ABI in ``include/upslam.h`` (argument marshalling only).

Loading fails loudly when ``libupslam.so`` is missing or cannot be built: there
is no CPU fallback anywhere in the product path.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libupslam.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_DEGENERATE, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_CAPACITY = range(8)
LOSS_L2, LOSS_L1 = 0, 1
F32, F16 = 0, 1


class Pano(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("el_top", ctypes.c_float),
                ("s_az", ctypes.c_float), ("s_el", ctypes.c_float), ("r_min", ctypes.c_float),
                ("r_max", ctypes.c_float)]


class NormalParams(ctypes.Structure):
    _fields_ = [("jump_rel", ctypes.c_float), ("jump_abs", ctypes.c_float), ("min_cross", ctypes.c_float)]


class IcpParams(ctypes.Structure):
    _fields_ = [("d_max", ctypes.c_float), ("cos_theta_max", ctypes.c_float), ("max_iters", ctypes.c_int32),
                ("min_inliers", ctypes.c_int32), ("eps_rot", ctypes.c_double), ("eps_trans", ctypes.c_double),
                ("pivot_eps", ctypes.c_double), ("loss", ctypes.c_int32), ("loss_delta", ctypes.c_float),
                ("coarse_iters", ctypes.c_int32), ("d_max_fine", ctypes.c_float)]


class FuseParams(ctypes.Structure):
    _fields_ = [("d_max", ctypes.c_float), ("cos_theta_max", ctypes.c_float), ("w_max", ctypes.c_float),
                ("accept_quality", ctypes.c_float)]


class IcpStats(ctypes.Structure):
    _fields_ = [("A", ctypes.c_double * 21), ("b", ctypes.c_double * 6), ("sse", ctypes.c_double),
                ("inliers", ctypes.c_int64), ("valid", ctypes.c_int64), ("status", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("xi", ctypes.c_double * 6), ("iters", ctypes.c_int32),
                ("accepted", ctypes.c_int32)]


class Sweep(ctypes.Structure):
    _fields_ = [("pano", Pano), ("d_pix", ctypes.c_void_p), ("d_nrm", ctypes.c_void_p),
                ("nrm_precision", ctypes.c_int32)]


class Keyframe(ctypes.Structure):
    _fields_ = [("pano", Pano), ("d_depth", ctypes.c_void_p), ("d_nw", ctypes.c_void_p),
                ("precision", ctypes.c_int32), ("d_dirs", ctypes.c_void_p)]


class SweepBuffers(ctypes.Structure):
    _fields_ = [("pano", Pano), ("d_zbuf", ctypes.c_void_p), ("d_depth", ctypes.c_void_p), ("d_idx", ctypes.c_void_p),
                ("d_pix", ctypes.c_void_p), ("d_nrm", ctypes.c_void_p), ("nrm_precision", ctypes.c_int32)]


class BatchTiles(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("chunk", ctypes.c_int32)]


class AtrousParams(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("sigma_n", ctypes.c_float), ("sigma_x", ctypes.c_float)]


STATS_BYTES = ctypes.sizeof(IcpStats)
KEYFRAME_BYTES = ctypes.sizeof(Keyframe)
_P = ctypes.POINTER
_vp = ctypes.c_void_p

# name -> (restype, argtypes); every entry point declared in include/upslam.h
SIGNATURES = {
    "upslam_pano_dirs_floats": (ctypes.c_size_t, [_P(Pano)]),
    "upslam_pano_dirs": (ctypes.c_int, [_P(Pano), _vp, _vp]),
    "upslam_project": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _P(Pano), _vp, _vp, _vp, _vp, _vp]),
    "upslam_unproject": (ctypes.c_int, [_vp, _P(Pano), _vp, _vp, _vp]),
    "upslam_normals": (ctypes.c_int, [_vp, _vp, _P(Pano), _P(NormalParams), _vp, ctypes.c_int32, _vp]),
    "upslam_atrous_normals": (ctypes.c_int, [_P(Pano), _vp, _vp, _vp, _vp, ctypes.c_int32, _P(AtrousParams), _vp]),
    "upslam_icp_workspace_bytes": (ctypes.c_size_t, [_P(Keyframe)]),
    "upslam_icp_step": (ctypes.c_int, [_P(Keyframe), _P(Sweep), _vp, _P(IcpParams), _vp, _vp, ctypes.c_size_t, _vp]),
    "upslam_icp": (ctypes.c_int, [_P(Keyframe), _P(Sweep), _vp, _P(IcpParams), _vp, _vp, ctypes.c_size_t, _vp]),
    "upslam_fuse": (ctypes.c_int, [_P(Keyframe), _P(Sweep), _vp, _P(FuseParams), _vp, _vp, _vp]),
    "upslam_track": (ctypes.c_int, [_P(Keyframe), _P(Sweep), _vp, _vp, _vp, ctypes.c_int32, _P(IcpParams),
                                    _P(FuseParams), _vp, _vp, ctypes.c_size_t, _vp, _vp]),
    "upslam_track_scan": (ctypes.c_int, [_P(Keyframe), _vp, ctypes.c_int32, _P(SweepBuffers), _P(NormalParams), _vp,
                                         _vp, _vp, ctypes.c_int32, _P(IcpParams), _P(FuseParams), _vp, _vp,
                                         ctypes.c_size_t, _vp, _vp]),
    "upslam_register": (ctypes.c_int, [_P(Keyframe), _P(Sweep), _vp, _vp, _vp, ctypes.c_int32, _P(IcpParams), _vp, _vp,
                                       ctypes.c_size_t, _vp]),
    "upslam_icp_noalloc_capacity_bytes": (ctypes.c_size_t, []),
    "upslam_icp_noalloc": (ctypes.c_int, [_P(Keyframe), _P(Sweep), _vp, _P(IcpParams), _vp, _vp]),
    "upslam_icp_wait_probe": (ctypes.c_int, [_P(Keyframe), _P(Sweep), _vp, _P(IcpParams), _vp, _vp, ctypes.c_size_t,
                                             ctypes.c_longlong, _vp]),
    "upslam_predict_pose": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "upslam_update_motion": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "upslam_icp_batched_workspace_bytes": (ctypes.c_size_t, [_P(Keyframe), ctypes.c_int32, ctypes.c_int32,
                                                             _P(BatchTiles)]),
    "upslam_icp_batched": (ctypes.c_int, [_vp, _P(Keyframe), ctypes.c_int32, _P(Sweep), ctypes.c_int32, _vp,
                                          _P(IcpParams), _vp, _vp, ctypes.c_size_t, _P(BatchTiles), _vp]),
    "upslam_grid_score": (ctypes.c_int, [_P(Keyframe), _P(Sweep), _vp, ctypes.c_int32, ctypes.c_int32, _P(IcpParams),
                                         _vp, _vp, _vp, _vp]),
    "upslam_grid_candidates": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp]),
    "upslam_consistency_workspace_bytes": (ctypes.c_size_t, [_P(Keyframe), _P(Keyframe)]),
    "upslam_keyframe_consistency": (ctypes.c_int, [_P(Keyframe), _P(Keyframe), _vp, ctypes.c_float, ctypes.c_float,
                                                   _vp, ctypes.c_size_t, _vp, _vp]),
    "upslam_cnn_param_count": (ctypes.c_size_t, []),
    "upslam_cnn_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int32]),
    "upslam_cnn_error_offset": (ctypes.c_size_t, [ctypes.c_int32]),
    "upslam_cnn_workspace_layout": (ctypes.c_size_t, [ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "upslam_cnn_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp, ctypes.c_size_t, _vp]),
    "upslam_cnn_forward_wait_probe": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp, ctypes.c_size_t,
                                                     ctypes.c_ulonglong, _vp]),
    "upslam_cnn_backward": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t,
                                           _vp]),
    "upslam_cnn_adam": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_float, _vp]),
    "upslam_downsample": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _P(Pano), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_float, _vp, ctypes.c_int32, ctypes.c_int32, _vp]),
    "upslam_se3_exp": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp]),
    "upslam_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "upslam_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


class UpslamError(RuntimeError):
    def __init__(self, fn: str, code: int):
        msg = lib().upslam_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{fn} failed: {msg} (status {code})")
        self.code = code


def lib(build_if_missing: bool = True):
    """The loaded library; builds it with nvcc when absent, raises when that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2101_00585_gb300.build.build()")
            from . import build as _build
            _build.build()
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def check(fn: str, code: int) -> None:
    if code != OK:
        raise UpslamError(fn, code)
