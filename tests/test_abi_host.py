"""Host-side checks of the C ABI (no GPU needed): exports and argument validation."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

import paper_2101_00585_gb300 as up
from paper_2101_00585_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "upslam.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(upslam_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    L = up.lib()
    names = declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(_abi.SIGNATURES), set(names) - set(_abi.SIGNATURES)
    assert L.upslam_version().startswith(b"upslam-gb300")


def test_status_strings():
    L = up.lib()
    for code in range(7):
        assert L.upslam_status_string(code)
    assert L.upslam_status_string(99) == b"unknown status"


def _pano(rows=4, cols=8):
    return _abi.Pano(rows, cols, 0.5, cols / 6.283185307, rows / 1.0, 0.1, 100.0)


def test_invalid_arguments_are_rejected_on_the_host():
    """Bad arguments return INVALID_ARG before any CUDA call (safe without a GPU)."""
    L = up.lib()
    pp = _pano()
    bad = _abi.Pano(0, 8, 0.5, 1.0, 1.0, 0.1, 100.0)
    fake = ctypes.c_void_p(256)
    assert L.upslam_project(fake, 10, None, ctypes.byref(bad), fake, fake, fake, None, None) == _abi.ERR_INVALID_ARG
    assert L.upslam_project(None, 10, None, ctypes.byref(pp), fake, fake, fake, None, None) == _abi.ERR_INVALID_ARG
    assert L.upslam_project(fake, -1, None, ctypes.byref(pp), fake, fake, fake, None, None) == _abi.ERR_INVALID_ARG
    misaligned = ctypes.c_void_p(256 + 4)
    assert L.upslam_project(misaligned, 10, None, ctypes.byref(pp), fake, fake, fake, None,
                            None) == _abi.ERR_INVALID_ARG
    npar = _abi.NormalParams(0.05, 0.1, 1e-4)
    assert L.upslam_normals(fake, fake, ctypes.byref(pp), ctypes.byref(npar), fake, 7, None) == _abi.ERR_INVALID_ARG
    assert L.upslam_pano_dirs(ctypes.byref(bad), fake, None) == _abi.ERR_INVALID_ARG
    assert L.upslam_pano_dirs_floats(ctypes.byref(bad)) == 0
    assert L.upslam_pano_dirs_floats(ctypes.byref(pp)) == 2 * 4 + 2 * 8
    ks = _abi.Keyframe(pp, 256, 256, 0, 256)
    ss = _abi.Sweep(pp, 256, 256, 0)
    ip = _abi.IcpParams(0.5, 0.86, 10, 6, 1e-6, 1e-6, 1e-12)
    ws = int(L.upslam_icp_workspace_bytes(ctypes.byref(ks)))
    assert ws >= 256
    # workspace too small / stats missing / bad precision
    assert L.upslam_icp_step(ctypes.byref(ks), ctypes.byref(ss), fake, ctypes.byref(ip), fake, fake, 16,
                             None) == _abi.ERR_INVALID_ARG
    assert L.upslam_icp(ctypes.byref(ks), ctypes.byref(ss), fake, ctypes.byref(ip), None, fake, ws,
                        None) == _abi.ERR_INVALID_ARG
    ks_bad = _abi.Keyframe(pp, 256, 256, 5, 256)
    assert L.upslam_icp_step(ctypes.byref(ks_bad), ctypes.byref(ss), fake, ctypes.byref(ip), fake, fake, ws,
                             None) == _abi.ERR_INVALID_ARG
    fp = _abi.FuseParams(0.2, 0.86, 0.5, 0.1)  # w_max < 1
    assert L.upslam_fuse(ctypes.byref(ks), ctypes.byref(ss), fake, ctypes.byref(fp), None, fake,
                         None) == _abi.ERR_INVALID_ARG
    # unknown loss, or the absolute error without a positive delta
    # ... or a coarse-to-fine gate with a negative step count or no fine gate
    for bad_ip in (_abi.IcpParams(0.5, 0.86, 10, 6, 1e-6, 1e-6, 1e-12, 2, 0.01),
                   _abi.IcpParams(0.5, 0.86, 10, 6, 1e-6, 1e-6, 1e-12, 1, 0.0),
                   _abi.IcpParams(0.5, 0.86, 10, 6, 1e-6, 1e-6, 1e-12, 0, 0.01, -1, 0.5),
                   _abi.IcpParams(0.5, 0.86, 10, 6, 1e-6, 1e-6, 1e-12, 0, 0.01, 5, 0.0)):
        assert L.upslam_icp(ctypes.byref(ks), ctypes.byref(ss), fake, ctypes.byref(bad_ip), fake, fake, ws,
                            None) == _abi.ERR_INVALID_ARG
    assert L.upslam_predict_pose(None, None, fake, None) == _abi.ERR_INVALID_ARG
    assert L.upslam_update_motion(fake, None, fake, None) == _abi.ERR_INVALID_ARG
    ap = _abi.AtrousParams(3, 0.5, 0.02)
    f2 = [ctypes.c_void_p(256 * i) for i in (1, 2, 3, 4)]
    assert L.upslam_atrous_normals(ctypes.byref(bad), f2[0], f2[1], f2[2], f2[3], 0, ctypes.byref(ap),
                                   None) == _abi.ERR_INVALID_ARG
    assert L.upslam_atrous_normals(ctypes.byref(pp), f2[0], f2[1], f2[1], f2[3], 0, ctypes.byref(ap),
                                   None) == _abi.ERR_INVALID_ARG  # input aliases output
    assert L.upslam_atrous_normals(ctypes.byref(pp), f2[0], f2[1], f2[2], None, 0, ctypes.byref(ap),
                                   None) == _abi.ERR_INVALID_ARG  # two or more levels need scratch
    assert L.upslam_atrous_normals(ctypes.byref(pp), f2[0], f2[1], f2[2], f2[3], 0,
                                   ctypes.byref(_abi.AtrousParams(4, 0.5, 0.02)), None) == _abi.ERR_INVALID_ARG
    assert L.upslam_atrous_normals(ctypes.byref(pp), f2[0], f2[1], f2[2], f2[3], 0,
                                   ctypes.byref(_abi.AtrousParams(2, float("nan"), 0.02)), None) == _abi.ERR_INVALID_ARG


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the header structs have the sizes and field offsets a C compiler gives them."""
    import subprocess
    mirrors = {"upslam_pano": _abi.Pano, "upslam_normal_params": _abi.NormalParams,
               "upslam_icp_params": _abi.IcpParams, "upslam_fuse_params": _abi.FuseParams,
               "upslam_icp_stats": _abi.IcpStats, "upslam_sweep": _abi.Sweep, "upslam_keyframe": _abi.Keyframe,
               "upslam_atrous_params": _abi.AtrousParams, "upslam_batch_tiles": _abi.BatchTiles,
               "upslam_sweep_buffers": _abi.SweepBuffers}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "upslam.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(ln.split() for ln in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, cls in mirrors.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The package never imports the oracle and refuses to run without its library."""
    pkg = os.path.join(ROOT, "paper_2101_00585_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "upslam_oracle" not in src, f
    with pytest.raises(RuntimeError):
        saved = _abi._lib, _abi.LIB_PATH
        try:
            _abi._lib = None
            _abi.LIB_PATH = "/nonexistent/libupslam.so"
            _abi.lib(build_if_missing=False)
        finally:
            _abi._lib, _abi.LIB_PATH = saved


def test_cnn_workspace_and_error_word_offsets():
    """The pose network's workspace size grows with the batch and its error word is the last 256-byte block."""
    L = up.lib()
    assert L.upslam_cnn_workspace_bytes(0) == 0 and L.upslam_cnn_error_offset(0) == 0
    prev = 0
    for b in (1, 3, 64, 256):
        ws = L.upslam_cnn_workspace_bytes(b)
        off = L.upslam_cnn_error_offset(b)
        assert ws > prev and ws % 256 == 0
        assert off == ws - 256 and off % 256 == 0
        prev = ws


def test_fused_batched_and_added_entry_points_reject_bad_arguments():
    """The fused per-sweep launches, the batched form, the next rows and the pose network check their
    arguments on the host too: each bad call returns INVALID_ARG before any CUDA call."""
    L = up.lib()
    INV = _abi.ERR_INVALID_ARG
    pp = _pano()
    fake = ctypes.c_void_p(256)
    ks = _abi.Keyframe(pp, 256, 256, 0, 256)
    ss = _abi.Sweep(pp, 256, 256, 0)
    ip = _abi.IcpParams(0.5, 0.86, 10, 6, 1e-6, 1e-6, 1e-12)
    fp = _abi.FuseParams(0.2, 0.86, 10.0, 0.3)
    ws = int(L.upslam_icp_workspace_bytes(ctypes.byref(ks)))
    K, S, I, F = (ctypes.byref(x) for x in (ks, ss, ip, fp))
    # motion prior: mode out of range, or a mode that needs a buffer that is missing
    for prior, prev, motion in ((3, fake, fake), (-1, fake, fake), (1, None, fake), (2, fake, None)):
        assert L.upslam_register(K, S, prev, motion, fake, prior, I, fake, fake, ws, None) == INV
        assert L.upslam_track(K, S, prev, motion, fake, prior, I, F, fake, fake, ws, fake, None) == INV
    # track: a bad keyframe-update parameter, no keyframe z-buffer, no iterations
    assert L.upslam_track(K, S, None, None, fake, 0, I, ctypes.byref(_abi.FuseParams(0.2, 0.86, 0.5, 0.3)), fake,
                          fake, ws, fake, None) == INV
    assert L.upslam_track(K, S, None, None, fake, 0, I, F, fake, fake, ws, None, None) == INV
    assert L.upslam_track(K, S, None, None, fake, 0, ctypes.byref(_abi.IcpParams(0.5, 0.86, 0, 6, 1e-6, 1e-6, 1e-12)),
                          F, fake, fake, ws, fake, None) == INV
    # whole-sweep launch: points missing, buffers missing, a misaligned point array
    sb = _abi.SweepBuffers(pp, 256, 256, 256, 256, 256, 0)
    npar = _abi.NormalParams(0.05, 0.1, 1e-4)
    SB, NP = ctypes.byref(sb), ctypes.byref(npar)
    assert L.upslam_track_scan(K, None, 10, SB, NP, None, None, fake, 0, I, F, fake, fake, ws, fake, None) == INV
    assert L.upslam_track_scan(K, fake, 10, None, NP, None, None, fake, 0, I, F, fake, fake, ws, fake, None) == INV
    assert L.upslam_track_scan(K, ctypes.c_void_p(260), 10, SB, NP, None, None, fake, 0, I, F, fake, fake, ws, fake,
                               None) == INV
    assert L.upslam_track_scan(K, fake, -1, SB, NP, None, None, fake, 0, I, F, fake, fake, ws, fake, None) == INV
    # the allocation-free form needs its stats record
    assert L.upslam_icp_noalloc(K, S, fake, I, None, None) == INV
    # batched form: no keyframes, no hypotheses, too many keyframes
    tiles = ctypes.byref(_abi.BatchTiles(512, 512))
    for n_kf, n_hyp in ((0, 8), (4, 0), (257, 1)):
        assert L.upslam_icp_batched(fake, K, n_kf, S, n_hyp, fake, I, fake, fake, 1 << 20, tiles, None) == INV
    # grid search: no candidates, a zero stride, one candidate past the documented limit (65535 CTA rows of
    # 32), a negative count
    assert L.upslam_grid_score(K, S, fake, 0, 4, I, fake, fake, fake, None) == INV
    assert L.upslam_grid_score(K, S, fake, 9, 0, I, fake, fake, fake, None) == INV
    assert L.upslam_grid_score(K, S, fake, 2097121, 4, I, fake, fake, fake, None) == INV
    assert L.upslam_grid_candidates(fake, fake, -1, fake, None) == INV
    assert L.upslam_grid_candidates(fake, fake, 0, fake, None) == _abi.OK  # nothing to do, nothing launched
    # consistency: a keyframe against itself in place, a negative tolerance, a misaligned workspace
    kb = _abi.Keyframe(pp, 512, 512, 0, 512)
    KB = ctypes.byref(kb)
    cws = int(L.upslam_consistency_workspace_bytes(K, KB))
    assert L.upslam_keyframe_consistency(K, K, fake, 0.05, 0.2, fake, cws, None, None) == INV
    assert L.upslam_keyframe_consistency(K, KB, fake, -0.05, 0.2, fake, cws, None, None) == INV
    assert L.upslam_keyframe_consistency(K, KB, fake, 0.05, 0.2, ctypes.c_void_p(264), cws, None, None) == INV
    assert L.upslam_keyframe_consistency(K, KB, fake, 0.05, 0.2, fake, 0, None, None) == INV
    # pose network: an empty batch, a misaligned workspace, a missing loss, Adam before step 1
    nws = int(L.upslam_cnn_workspace_bytes(4))
    assert L.upslam_cnn_forward(fake, fake, 0, fake, fake, nws, None) == INV
    assert L.upslam_cnn_forward(fake, fake, 4, fake, ctypes.c_void_p(264), nws, None) == INV
    assert L.upslam_cnn_backward(fake, fake, 4, fake, fake, fake, fake, None, fake, nws, None) == INV
    assert L.upslam_cnn_adam(fake, fake, fake, fake, 0, ctypes.c_float(1e-3), None) == INV
    # network input: cells that do not divide the panorama, a non-positive depth scale, a bad precision
    big = _abi.Pano(64, 256, 0.5, 256 / 6.283185307, 64.0, 0.1, 100.0)
    BP = ctypes.byref(big)
    assert L.upslam_downsample(fake, fake, 0, BP, 60, 256, ctypes.c_float(20.0), fake, 8, 0, None) == INV
    assert L.upslam_downsample(fake, fake, 0, BP, 64, 256, ctypes.c_float(0.0), fake, 8, 0, None) == INV
    assert L.upslam_downsample(fake, fake, 3, BP, 64, 256, ctypes.c_float(20.0), fake, 8, 0, None) == INV
    assert L.upslam_downsample(fake, fake, 0, BP, 64, 256, ctypes.c_float(20.0), fake, 8, 5, None) == INV
    # twists to poses, and keyframe points
    assert L.upslam_se3_exp(fake, -1, fake, None) == INV
    assert L.upslam_se3_exp(fake, 0, fake, None) == _abi.OK
    assert L.upslam_unproject(fake, ctypes.byref(pp), fake, ctypes.c_void_p(264), None) == INV
