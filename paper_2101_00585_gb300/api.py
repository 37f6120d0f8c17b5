"""Python binding of the UPSLAM hot path over torch CUDA tensors.

Argument marshalling only: every step runs in ``libupslam.so`` kernels on the
current torch CUDA stream.  torch provides device memory and streams.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import torch

from . import _abi

F32, F16 = _abi.F32, _abi.F16


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _p(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("expected a CUDA tensor")


def pano_struct(p) -> _abi.Pano:
    """C panorama struct from an object with rows, cols, el_top, s_az, s_el, r_min, r_max."""
    f = lambda x: float(torch.tensor(float(x), dtype=torch.float32).item())  # noqa: E731  (round to FP32)
    return _abi.Pano(int(p.rows), int(p.cols), f(p.el_top), f(p.s_az), f(p.s_el), f(p.r_min), f(p.r_max))


@dataclass
class Params:
    """Thresholds the paper leaves open; these values are this implementation's readings."""
    jump_rel: float = 0.05
    jump_abs: float = 0.1
    min_cross: float = 1e-4
    d_max: float = 0.5
    cos_theta_max: float = math.cos(math.radians(30.0))
    max_iters: int = 15
    min_inliers: int = 6
    eps_rot: float = 1e-6
    eps_trans: float = 1e-6
    pivot_eps: float = 1e-12
    # Eq. 1's |.|: LOSS_L2 squares the point-to-plane error (Gauss-Newton); LOSS_L1 minimises it as
    # printed by IRLS with weights 1 / max(|r|, loss_delta)
    loss: int = 0
    loss_delta: float = 0.01
    # coarse-to-fine Omega gate: the first coarse_iters steps of a multi-step call use d_max, later
    # ones d_max_fine (0 steps: d_max throughout)
    coarse_iters: int = 0
    d_max_fine: float = 0.5
    fuse_d_max: float = 0.2
    fuse_cos_theta_max: float = math.cos(math.radians(30.0))
    w_max: float = 10.0
    accept_quality: float = 0.1
    # edge-avoiding a-trous smoothing of the sweep normals (Sec. III-A); 0 levels = off
    atrous_levels: int = 0
    atrous_sigma_n: float = 0.5
    atrous_sigma_x: float = 0.02

    def normal(self):
        return _abi.NormalParams(self.jump_rel, self.jump_abs, self.min_cross)

    def icp(self):
        return _abi.IcpParams(self.d_max, self.cos_theta_max, self.max_iters, self.min_inliers, self.eps_rot,
                              self.eps_trans, self.pivot_eps, self.loss, self.loss_delta, self.coarse_iters,
                              self.d_max_fine)

    def fuse(self):
        return _abi.FuseParams(self.fuse_d_max, self.fuse_cos_theta_max, self.w_max, self.accept_quality)

    def atrous(self):
        return _abi.AtrousParams(self.atrous_levels, self.atrous_sigma_n, self.atrous_sigma_x)


def empty_zbuf(npx: int, device) -> torch.Tensor:
    """z-buffer scratch in its required resting state (all bits set)."""
    return torch.full((npx,), -1, dtype=torch.int64, device=device)


def identity_pose(device) -> torch.Tensor:
    T = torch.zeros(12, dtype=torch.float64, device=device)
    T[0] = T[5] = T[10] = 1.0
    return T


# ----------------------------------------------------------------------------- single calls

def pano_dirs(pp, device="cuda") -> torch.Tensor:
    ps = pano_struct(pp)
    n = _abi.lib().upslam_pano_dirs_floats(ctypes.byref(ps))
    out = torch.empty(n, dtype=torch.float32, device=device)
    _abi.check("upslam_pano_dirs", _abi.lib().upslam_pano_dirs(ctypes.byref(ps), _p(out), _stream()))
    return out


def project(pts4: torch.Tensor, pp, pose: torch.Tensor | None = None, zbuf: torch.Tensor | None = None,
            with_points: bool = True):
    """Sec. III-A projection -> (depth [H,W] f32, idx [H,W] i32, pix [H,W,4] f32 or None)."""
    _require_cuda(pts4, pose, zbuf)
    pts4 = pts4.contiguous()
    assert pts4.dtype == torch.float32 and pts4.shape[-1] == 4
    H, W = int(pp.rows), int(pp.cols)
    dev = pts4.device
    if zbuf is None:
        zbuf = empty_zbuf(H * W, dev)
    depth = torch.empty((H, W), dtype=torch.float32, device=dev)
    idx = torch.empty((H, W), dtype=torch.int32, device=dev)
    pix = torch.empty((H, W, 4), dtype=torch.float32, device=dev) if with_points else None
    ps = pano_struct(pp)
    _abi.check("upslam_project", _abi.lib().upslam_project(_p(pts4), pts4.shape[0], _p(pose), ctypes.byref(ps),
                                                           _p(zbuf), _p(depth), _p(idx), _p(pix), _stream()))
    return depth, idx, pix


def unproject(depth: torch.Tensor, pp, dirs: torch.Tensor) -> torch.Tensor:
    _require_cuda(depth, dirs)
    pix = torch.empty(depth.shape + (4,), dtype=torch.float32, device=depth.device)
    ps = pano_struct(pp)
    _abi.check("upslam_unproject", _abi.lib().upslam_unproject(_p(depth.contiguous()), ctypes.byref(ps), _p(dirs),
                                                               _p(pix), _stream()))
    return pix


def normals(pix: torch.Tensor, depth: torch.Tensor, pp, params: Params = Params(), precision: int = F32):
    """Sec. III-A cross-product normals -> [H,W,4] (nx, ny, nz, valid) in f32 or f16."""
    _require_cuda(pix, depth)
    dt = torch.float32 if precision == F32 else torch.float16
    out = torch.empty(depth.shape + (4,), dtype=dt, device=depth.device)
    ps = pano_struct(pp)
    npar = params.normal()
    _abi.check("upslam_normals", _abi.lib().upslam_normals(_p(pix.contiguous()), _p(depth.contiguous()),
                                                           ctypes.byref(ps), ctypes.byref(npar), _p(out), precision,
                                                           _stream()))
    return out


def atrous_normals(pix: torch.Tensor, nrm: torch.Tensor, pp, params: Params = Params(), precision: int = F32):
    """Edge-avoiding a-trous smoothing (Sec. III-A) of a [H,W,4] normal image -> a new [H,W,4] image."""
    _require_cuda(pix, nrm)
    out = torch.empty_like(nrm)
    tmp = torch.empty_like(nrm)
    ps = pano_struct(pp)
    ap = params.atrous()
    _abi.check("upslam_atrous_normals",
               _abi.lib().upslam_atrous_normals(ctypes.byref(ps), _p(pix.contiguous()), _p(nrm.contiguous()), _p(out),
                                                _p(tmp), precision, ctypes.byref(ap), _stream()))
    return out


class SweepFrame:
    """Device buffers of one sweep panorama: pixel points and normals."""

    def __init__(self, pp, device="cuda", precision: int = F32):
        self.pp = pp
        self.precision = precision
        H, W = int(pp.rows), int(pp.cols)
        self.zbuf = empty_zbuf(H * W, device)
        self.depth = torch.zeros((H, W), dtype=torch.float32, device=device)
        self.idx = torch.zeros((H, W), dtype=torch.int32, device=device)
        self.pix = torch.zeros((H, W, 4), dtype=torch.float32, device=device)
        self.nrm = torch.zeros((H, W, 4), dtype=torch.float32 if precision == F32 else torch.float16, device=device)
        self._raw = self._tmp = None  # unsmoothed normals and a-trous scratch, allocated on first use
        self._ps = pano_struct(pp)

    def struct(self) -> _abi.Sweep:
        return _abi.Sweep(self._ps, self.pix.data_ptr(), self.nrm.data_ptr(), self.precision)

    def buffers(self) -> _abi.SweepBuffers:
        """The buffers upslam_track_scan writes (projection, resolve, normals)."""
        return _abi.SweepBuffers(self._ps, self.zbuf.data_ptr(), self.depth.data_ptr(), self.idx.data_ptr(),
                                 self.pix.data_ptr(), self.nrm.data_ptr(), self.precision)

    def load(self, pts4: torch.Tensor, params: Params) -> None:
        """project + normals (+ a-trous smoothing when params.atrous_levels > 0) for a scan already on
        the device (float4 points)."""
        L = _abi.lib()
        s = _stream()
        _abi.check("upslam_project", L.upslam_project(_p(pts4), pts4.shape[0], None, ctypes.byref(self._ps),
                                                      _p(self.zbuf), _p(self.depth), _p(self.idx), _p(self.pix), s))
        npar = params.normal()
        levels = int(params.atrous_levels)
        if levels > 0 and self._raw is None:
            self._raw = torch.zeros_like(self.nrm)
            self._tmp = torch.zeros_like(self.nrm)
        dst = self._raw if levels > 0 else self.nrm
        _abi.check("upslam_normals", L.upslam_normals(_p(self.pix), _p(self.depth), ctypes.byref(self._ps),
                                                      ctypes.byref(npar), _p(dst), self.precision, s))
        if levels > 0:
            ap = params.atrous()
            _abi.check("upslam_atrous_normals",
                       L.upslam_atrous_normals(ctypes.byref(self._ps), _p(self.pix), _p(self._raw), _p(self.nrm),
                                               _p(self._tmp), self.precision, ctypes.byref(ap), s))

    def set(self, pix: torch.Tensor, nrm: torch.Tensor) -> None:
        """Use given pixel points / normals (e.g. test inputs) instead of computing them."""
        self.pix.copy_(pix)
        self.nrm.copy_(nrm)


class KeyframeBuffer:
    """Device keyframe panorama: depth, normals + sample count, direction table."""

    def __init__(self, pp, device="cuda", precision: int = F32):
        self.pp = pp
        self.precision = precision
        H, W = int(pp.rows), int(pp.cols)
        self.depth = torch.zeros((H, W), dtype=torch.float32, device=device)
        self.nw = torch.zeros((H, W, 4), dtype=torch.float32 if precision == F32 else torch.float16, device=device)
        self.dirs = pano_dirs(pp, device)
        self.zbuf = empty_zbuf(H * W, device)
        self._ps = pano_struct(pp)

    def struct(self) -> _abi.Keyframe:
        return _abi.Keyframe(self._ps, self.depth.data_ptr(), self.nw.data_ptr(), self.precision,
                             self.dirs.data_ptr())

    def clear(self) -> None:
        self.depth.zero_()
        self.nw.zero_()

    def set(self, depth: torch.Tensor, nw: torch.Tensor) -> None:
        self.depth.copy_(depth)
        self.nw.copy_(nw)

    def save(self, path: str) -> None:
        """Write the keyframe (geometry, depth, normals and counts) to a ``.npz`` file."""
        import numpy as np
        pp = self.pp
        np.savez(path, rows=int(pp.rows), cols=int(pp.cols), el_top=float(pp.el_top), s_az=float(pp.s_az),
                 s_el=float(pp.s_el), r_min=float(pp.r_min), r_max=float(pp.r_max), precision=int(self.precision),
                 depth=self.depth.cpu().numpy(), nw=self.nw.cpu().numpy())

    @classmethod
    def load(cls, path: str, device="cuda") -> "KeyframeBuffer":
        """A keyframe written by ``save``, on ``device``."""
        import numpy as np
        from types import SimpleNamespace
        z = np.load(path)
        pp = SimpleNamespace(**{k: z[k].item() for k in ("rows", "cols", "el_top", "s_az", "s_el", "r_min", "r_max")})
        kf = cls(pp, device, int(z["precision"]))
        kf.set(torch.from_numpy(z["depth"]).to(device), torch.from_numpy(z["nw"]).to(device))
        return kf


class IcpState:
    """Device-resident pose, stats and workspace for one registration problem."""

    def __init__(self, kf: KeyframeBuffer, device="cuda"):
        L = _abi.lib()
        ks = kf.struct()
        self.ws_bytes = int(L.upslam_icp_workspace_bytes(ctypes.byref(ks)))
        self.ws = torch.zeros(self.ws_bytes, dtype=torch.uint8, device=device)
        self.stats = torch.zeros(_abi.STATS_BYTES, dtype=torch.uint8, device=device)
        self.pose = identity_pose(device)

    def read_stats(self) -> dict:
        raw = bytes(self.stats.cpu().numpy())
        st = _abi.IcpStats.from_buffer_copy(raw)
        return {"A": list(st.A), "b": list(st.b), "sse": st.sse, "inliers": st.inliers, "valid": st.valid,
                "status": st.status, "converged": st.converged, "xi": list(st.xi), "iters": st.iters,
                "accepted": st.accepted}


def icp_step(kf: KeyframeBuffer, sw: SweepFrame, state: IcpState, params: Params = Params()) -> None:
    ks, ss, ip = kf.struct(), sw.struct(), params.icp()
    _abi.check("upslam_icp_step", _abi.lib().upslam_icp_step(ctypes.byref(ks), ctypes.byref(ss), _p(state.pose),
                                                             ctypes.byref(ip), _p(state.stats), _p(state.ws),
                                                             state.ws_bytes, _stream()))


def icp(kf: KeyframeBuffer, sw: SweepFrame, state: IcpState, params: Params = Params()) -> None:
    ks, ss, ip = kf.struct(), sw.struct(), params.icp()
    _abi.check("upslam_icp", _abi.lib().upslam_icp(ctypes.byref(ks), ctypes.byref(ss), _p(state.pose),
                                                   ctypes.byref(ip), _p(state.stats), _p(state.ws), state.ws_bytes,
                                                   _stream()))


def fuse(kf: KeyframeBuffer, sw: SweepFrame, pose: torch.Tensor, params: Params = Params(),
         stats: torch.Tensor | None = None) -> None:
    ks, ss, fp = kf.struct(), sw.struct(), params.fuse()
    _abi.check("upslam_fuse", _abi.lib().upslam_fuse(ctypes.byref(ks), ctypes.byref(ss), _p(pose), ctypes.byref(fp),
                                                     _p(stats), _p(kf.zbuf), _stream()))


# ----------------------------------------------------------------------------- the per-sweep path

class Tracker:
    """Registers a stream of sweeps against keyframes and fuses them in (Sec. III).

    Everything stays on the device: the pose of the current sweep in the
    current keyframe (``state.pose``), the last inter-sweep motion, the
    registration record.  ``track`` launches project, normals, the motion
    prior, the persistent ICP and the keyframe update on the current stream
    with no host synchronisation.  ``new_keyframe`` starts a keyframe at the
    current sweep (its frame becomes the keyframe frame) by hole-filling an
    empty panorama.
    """

    def __init__(self, sweep_pano, kf_pano, params: Params = Params(), precision: int = F32, device="cuda",
                 constant_velocity: bool = True, fused: bool = True, front_fused: bool = True):
        self.params = params
        self.sw = SweepFrame(sweep_pano, device, precision)
        self.kf = KeyframeBuffer(kf_pano, device, precision)
        self.state = IcpState(self.kf, device)
        self.motion = identity_pose(device)
        self.prev = identity_pose(device)
        self.identity = identity_pose(device)
        self.constant_velocity = constant_velocity
        self.fused = fused
        # one launch per sweep (projection and normals inside the register + update launch); needs
        # `fused` and no a-trous smoothing, which runs as launches of its own between the two
        self.front_fused = front_fused and fused and int(params.atrous_levels) == 0
        self._ip, self._fp = params.icp(), params.fuse()
        self._np = params.normal()

    def new_keyframe(self, pts4: torch.Tensor | None = None, buffer: KeyframeBuffer | None = None,
                     consistency: bool = False) -> None:
        """Start a keyframe at the sweep in ``self.sw`` (loading ``pts4`` first if given).

        ``buffer``: an all-zero keyframe buffer to use from now on (for example one of a
        pre-allocated pool); without it the current buffer is cleared and reused.
        ``consistency`` (needs ``buffer``): run the mutual consistency check (Sec. III-C)
        between the keyframe being left and the new one; the new keyframe's pose in the old
        one is the last registered sweep pose.
        """
        if pts4 is not None:
            self.sw.load(pts4, self.params)
        old = self.kf
        if buffer is not None:
            self.kf = buffer
        else:
            if consistency:
                raise ValueError("the consistency check needs a separate buffer for the new keyframe")
            self.kf.clear()
        fuse(self.kf, self.sw, self.identity, self.params, None)
        if consistency:
            self.last_removed = keyframe_consistency(old, self.kf, self.state.pose)[0]
        self.prev.copy_(self.identity)

    # optional profiling hook: (recorder, stream, proj_events, icp_events, fuse_events); the recorder's
    # record(event, stream) is called around the three phases of track()
    timing = None

    def _mark(self, which: int, edge: int) -> None:
        tm = self.timing
        if tm is not None:
            tm[0].record(tm[2 + which][edge], tm[1])

    def track(self, pts4: torch.Tensor) -> None:
        """One sweep: project, normals, prior, ICP, keyframe update (all asynchronous)."""
        L = _abi.lib()
        s = _stream()
        if self.front_fused:
            # projection, normals, prior, ICP, motion update and keyframe update in one launch
            ks, sb = self.kf.struct(), self.sw.buffers()
            self._mark(0, 0)
            self._mark(0, 1)
            self._mark(1, 0)
            _abi.check("upslam_track_scan",
                       L.upslam_track_scan(ctypes.byref(ks), _p(pts4), pts4.shape[0], ctypes.byref(sb),
                                           ctypes.byref(self._np), _p(self.prev), _p(self.motion),
                                           _p(self.state.pose), 2 if self.constant_velocity else 1,
                                           ctypes.byref(self._ip), ctypes.byref(self._fp), _p(self.state.stats),
                                           _p(self.state.ws), self.state.ws_bytes, _p(self.kf.zbuf), s))
            self._mark(1, 1)
            self._mark(2, 0)
            self._mark(2, 1)
            return
        self._mark(0, 0)
        self.sw.load(pts4, self.params)
        self._mark(0, 1)
        ks, ss = self.kf.struct(), self.sw.struct()
        self._mark(1, 0)
        if self.fused:
            # prior + ICP + motion update + keyframe update in one persistent launch
            _abi.check("upslam_track", L.upslam_track(ctypes.byref(ks), ctypes.byref(ss), _p(self.prev),
                                                      _p(self.motion), _p(self.state.pose),
                                                      2 if self.constant_velocity else 1, ctypes.byref(self._ip),
                                                      ctypes.byref(self._fp), _p(self.state.stats), _p(self.state.ws),
                                                      self.state.ws_bytes, _p(self.kf.zbuf), s))
            self._mark(1, 1)
            self._mark(2, 0)
            self._mark(2, 1)
            return
        # prior + ICP + motion update in one launch; afterwards prev holds this sweep's pose
        _abi.check("upslam_register", L.upslam_register(ctypes.byref(ks), ctypes.byref(ss), _p(self.prev),
                                                        _p(self.motion), _p(self.state.pose),
                                                        2 if self.constant_velocity else 1, ctypes.byref(self._ip),
                                                        _p(self.state.stats), _p(self.state.ws), self.state.ws_bytes,
                                                        s))
        self._mark(1, 1)
        self._mark(2, 0)
        _abi.check("upslam_fuse", L.upslam_fuse(ctypes.byref(ks), ctypes.byref(ss), _p(self.state.pose),
                                                ctypes.byref(self._fp), _p(self.state.stats), _p(self.kf.zbuf), s))
        self._mark(2, 1)

    # kernels launched by one track() call: one (front_fused); else project (2), normals, one per
    # a-trous level, then one persistent register + update launch (fused), or register + fuse (2)
    @property
    def launches_per_track(self) -> int:
        if self.front_fused:
            return 1
        return (4 if self.fused else 6) + int(self.params.atrous_levels)
    # kernels launched by new_keyframe() (after loading): fuse (2)
    LAUNCHES_PER_NEW_KEYFRAME = 2


# ----------------------------------------------------------------------------- loop-closure grid search

def grid_candidates(center: torch.Tensor, xi: torch.Tensor) -> torch.Tensor:
    """Candidate poses exp(xi_i^) * center: center FP64 [12], xi FP32 [n, 6] -> FP64 [n, 12]."""
    _require_cuda(center, xi)
    xi = xi.contiguous().to(torch.float32)
    out = torch.empty((xi.shape[0], 12), dtype=torch.float64, device=xi.device)
    _abi.check("upslam_grid_candidates", _abi.lib().upslam_grid_candidates(_p(center.contiguous()), _p(xi),
                                                                           xi.shape[0], _p(out), _stream()))
    return out


def grid_score(kf: "KeyframeBuffer", sw: "SweepFrame", poses: torch.Tensor, params: Params = Params(),
               stride: int = 4):
    """Sec. III-C grid search: inlier counts of the candidates [n, 12] on the keyframe sampled every
    ``stride`` pixels -> (scores int64 [n], best int32 [1], best pose FP64 [12]), all on the device."""
    _require_cuda(poses)
    poses = poses.contiguous()
    n = poses.shape[0]
    scores = torch.empty(n, dtype=torch.int64, device=poses.device)
    best = torch.empty(1, dtype=torch.int32, device=poses.device)
    best_pose = torch.empty(12, dtype=torch.float64, device=poses.device)
    ks, ss, ip = kf.struct(), sw.struct(), params.icp()
    _abi.check("upslam_grid_score", _abi.lib().upslam_grid_score(ctypes.byref(ks), ctypes.byref(ss), _p(poses), n,
                                                                 int(stride), ctypes.byref(ip), _p(scores), _p(best),
                                                                 _p(best_pose), _stream()))
    return scores, best, best_pose


# ----------------------------------------------------------------------------- keyframe consistency

def keyframe_consistency(kf_a: "KeyframeBuffer", kf_b: "KeyframeBuffer", T_ab: torch.Tensor, rel: float = 0.05,
                         abs_m: float = 0.2):
    """Sec. III-C mutual consistency check between two keyframes (T_ab: pose of B in A, FP64 [12] on the
    device).  Samples of each keyframe that the other saw through are removed in place.
    -> (removed int64 [2] on the device, flags_a uint8 [Ha, Wa], flags_b uint8 [Hb, Wb])."""
    _require_cuda(T_ab)
    L = _abi.lib()
    ka, kb = kf_a.struct(), kf_b.struct()
    nbytes = int(L.upslam_consistency_workspace_bytes(ctypes.byref(ka), ctypes.byref(kb)))
    ws = torch.zeros(nbytes, dtype=torch.uint8, device=T_ab.device)
    removed = torch.zeros(2, dtype=torch.int64, device=T_ab.device)
    _abi.check("upslam_keyframe_consistency",
               L.upslam_keyframe_consistency(ctypes.byref(ka), ctypes.byref(kb), _p(T_ab.contiguous()), float(rel),
                                             float(abs_m), _p(ws), nbytes, _p(removed), _stream()))
    Ha, Wa = int(kf_a.pp.rows), int(kf_a.pp.cols)
    Hb, Wb = int(kf_b.pp.rows), int(kf_b.pp.cols)
    off_b = (Ha * Wa + 255) // 256 * 256
    return removed, ws[:Ha * Wa].view(Ha, Wa), ws[off_b:off_b + Hb * Wb].view(Hb, Wb)


# ----------------------------------------------------------------------------- batched registration

class Batch:
    """One sweep against several keyframes with several initial poses each, solved in one launch.

    Problem p = kf * n_hyp + h.  ``run(init_poses)`` registers all problems; the
    results are in ``poses`` ([n_prob, 12] FP64) and ``read_stats()``.
    """

    def __init__(self, sweep: SweepFrame, keyframes: list, n_hyp: int, tiles: tuple | None = None, device="cuda"):
        self.sw = sweep
        self.kfs = list(keyframes)
        self.n_kf, self.n_hyp = len(self.kfs), int(n_hyp)
        self.n_prob = self.n_kf * self.n_hyp
        arr = (_abi.Keyframe * self.n_kf)(*[k.struct() for k in self.kfs])
        self._host = arr
        raw = bytes(arr)
        self.d_table = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)
        self.set_tiles(tiles)
        self.poses = torch.zeros((self.n_prob, 12), dtype=torch.float64, device=device)
        self.stats = torch.zeros((self.n_prob, _abi.STATS_BYTES), dtype=torch.uint8, device=device)
        self.device = device

    def set_tiles(self, tiles):
        self.tiles = _abi.BatchTiles(*(tiles or (512, 512)))
        L = _abi.lib()
        self.ws_bytes = int(L.upslam_icp_batched_workspace_bytes(self._host, self.n_kf, self.n_hyp,
                                                                  ctypes.byref(self.tiles)))
        if getattr(self, "ws", None) is None or self.ws.numel() < self.ws_bytes:
            self.ws = torch.zeros(self.ws_bytes, dtype=torch.uint8, device=self.sw.pix.device)

    def _launch(self, params: Params) -> None:
        ip = params.icp()
        ss = self.sw.struct()
        _abi.check("upslam_icp_batched",
                   _abi.lib().upslam_icp_batched(_p(self.d_table), self._host, self.n_kf, ctypes.byref(ss), self.n_hyp,
                                                 _p(self.poses), ctypes.byref(ip), _p(self.stats), _p(self.ws),
                                                 self.ws_bytes, ctypes.byref(self.tiles), _stream()))

    def run(self, init_poses: torch.Tensor, params: Params = Params()) -> None:
        """Register every problem from ``init_poses`` ([n_prob, 12] FP64) in one launch (eager)."""
        self.poses.copy_(init_poses.reshape(self.n_prob, 12))
        self._launch(params)

    def capture(self, params: Params = Params()) -> None:
        """Record one whole batched registration as a CUDA graph: the copy of ``self.init`` (FP64
        [n_prob, 12], write the initial poses there) into ``poses`` and the persistent launch.
        ``replay()`` then runs it with no host work.  The tiles and params are fixed at capture."""
        self.init = torch.zeros_like(self.poses)
        s = torch.cuda.Stream(device=self.poses.device)
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.poses.copy_(self.init)
            self._launch(params)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g

    def replay(self) -> None:
        """Run the captured registration on the current stream (``capture`` first)."""
        self.graph.replay()

    def read_stats(self) -> list:
        raw = self.stats.cpu().numpy()
        out = []
        for p in range(self.n_prob):
            st = _abi.IcpStats.from_buffer_copy(bytes(raw[p]))
            out.append({"A": list(st.A), "b": list(st.b), "sse": st.sse, "inliers": st.inliers, "valid": st.valid,
                        "status": st.status, "converged": st.converged, "xi": list(st.xi), "iters": st.iters})
        return out
