"""GPU sweeps from the analytic scenes (FP32 CUDA ray caster; input generation only).

Used to make the many sweeps that training pairs for the pose-proposal network
need.  Same scenes, lidar models and noise model as the CPU caster, in FP32.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_raycast_cuda.so")
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "raycast_cuda.cu")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC",
                               "-shared", src, "-o", _SO])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp = ctypes.c_void_p
        lib.synth_cast_cuda.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_float, vp, vp]
        lib.synth_cast_cuda.restype = ctypes.c_int
        _lib = lib
    return _lib


class GpuCaster:
    """Batched sweeps of one scene with one lidar model on the current CUDA device."""

    def __init__(self, scene, lidar, device="cuda"):
        import torch
        self.torch = torch
        self.lidar = lidar
        self.device = device
        self.prims = torch.from_numpy(np.ascontiguousarray(scene.prims, np.float32)).to(device)
        self.nprims = int(scene.prims.shape[0])
        self.dirs_np = lidar.directions()
        self.dirs = torch.from_numpy(self.dirs_np.astype(np.float32)).to(device)

    def scans(self, poses, gen) -> "torch.Tensor":
        """[B, N, 4] float32 sweeps (x, y, z, valid) in sensor coordinates; noise from ``gen``."""
        torch = self.torch
        B, n = len(poses), self.dirs.shape[0]
        P = np.stack([np.asarray(p, np.float64) for p in poses])
        org = torch.from_numpy(P[:, :, 3].astype(np.float32)).to(self.device).contiguous()
        rot = torch.from_numpy(P[:, :, :3].reshape(B, 9).astype(np.float32)).to(self.device).contiguous()
        t = torch.empty((B, n), dtype=torch.float32, device=self.device)
        rc = _load().synth_cast_cuda(ctypes.c_void_p(self.prims.data_ptr()), self.nprims,
                                     ctypes.c_void_p(org.data_ptr()), ctypes.c_void_p(rot.data_ptr()),
                                     ctypes.c_void_p(self.dirs.data_ptr()), n, B, float(self.lidar.r_max * 1.2),
                                     ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc != 0:
            raise RuntimeError("GPU ray cast failed")
        valid = (t >= self.lidar.r_min) & (t <= self.lidar.r_max)
        rr = t + self.lidar.sigma * torch.randn(t.shape, generator=gen, device=self.device)
        valid &= torch.rand(t.shape, generator=gen, device=self.device) >= self.lidar.dropout
        valid &= (rr >= self.lidar.r_min) & (rr <= self.lidar.r_max)
        out = torch.zeros((B, n, 4), dtype=torch.float32, device=self.device)
        out[..., :3] = self.dirs[None] * rr[..., None]
        out[..., 3] = valid.float()
        out[..., :3] *= out[..., 3:4]
        return out
