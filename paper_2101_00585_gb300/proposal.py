"""Learned initial pose for ICP: training pairs, training and gated inference.

Not in the paper.  UPSLAM starts ICP from a zero-velocity or zero-acceleration prior (Sec. IV-F footnote), and a
large motion is left to the registration.  Here a small network predicts the keyframe-from-sweep pose of a pair;
ICP (Sec. III-B) refines it, and a gate on the ICP result falls back to the plain prior.

Every numerical step runs in libupslam kernels:
* the plain pipeline makes the pair: projection, normals, a keyframe hole-filled from a sweep, downsampling;
* the network runs forward, backward and Adam as BF16 tensor-core GEMMs with FP32 accumulation;
* twists become poses through ``upslam_se3_exp``;
* ICP runs through ``upslam_icp``.

This module only schedules the calls and draws the seeded pair geometry.

Pair geometry: the sweep pose is the keyframe pose times a motion D, with |t| <= 1 m and |omega| <= 30 deg.
The label is xi = log(D), and the loss weighs rotation (rad) x4 against translation (m).
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np
import torch

from . import _abi
from .api import KeyframeBuffer, Params, SweepFrame, IcpState, _p, _stream, fuse, identity_pose, icp

IN_H, IN_W, IN_C = 64, 256, 8
DEPTH_SCALE = 20.0
LOSS_W = (4.0, 4.0, 4.0, 1.0, 1.0, 1.0)
CHANNELS = (8, 32, 64, 128, 128)


# ----------------------------------------------------------------------------- SE(3) labels (host, FP64)

def se3_log(T: np.ndarray) -> np.ndarray:
    """xi = (omega, v) with exp(xi^) = T (rotation angle < pi)."""
    R, t = T[:, :3], T[:, 3]
    c = (np.trace(R) - 1.0) / 2.0
    s = 0.5 * np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    th = math.atan2(np.linalg.norm(s), c)
    if th < 1e-8:
        w = s
    else:
        w = s * (th / math.sin(th))
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    th2 = th * th
    if th < 1e-6:
        Vinv = np.eye(3) - 0.5 * W + W @ W / 12.0
    else:
        Vinv = np.eye(3) - 0.5 * W + (1.0 / th2) * (1.0 - (th * math.sin(th)) / (2.0 * (1.0 - math.cos(th)))) * (W @ W)
    return np.concatenate([w, Vinv @ t])


def random_motion(rng: np.random.Generator, max_t: float = 1.0, max_deg: float = 30.0):
    """A rigid motion with a uniform translation length <= max_t (mostly horizontal) and rotation <= max_deg."""
    d = rng.standard_normal(3)
    d[2] *= 0.3
    d /= np.linalg.norm(d)
    t = d * rng.uniform(0.0, max_t)
    ax = rng.standard_normal(3)
    ax[2] += 2.0 * np.sign(ax[2] if ax[2] != 0 else 1.0)  # yaw-dominated
    ax /= np.linalg.norm(ax)
    ang = math.radians(rng.uniform(0.0, max_deg))
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)
    return np.hstack([R, t[:, None]])


# ----------------------------------------------------------------------------- network

S2D_FEATURES = 128  # features of the first layer's 2x2 space-to-depth convolution (4 taps x 32 channels)


def s2d_feature_source(f: int) -> int:
    """The 3x3 feature (ky, kx, c) -> 8 (3 ky + kx) + c whose weight the library's first-layer GEMM holds at
    feature f = 32 (2 ty + tx) + 16 dy + 8 dx + c of its space-to-depth order, where (ky, kx) =
    (2 ty + dy - 1, 2 tx + dx - 1); -1 where ky or kx is -1 (a feature the convolution never reads)."""
    tap, dy, dx, c = f >> 5, (f >> 4) & 1, (f >> 3) & 1, f & 7
    ky, kx = 2 * (tap >> 1) + dy - 1, 2 * (tap & 1) + dx - 1
    return -1 if ky < 0 or kx < 0 else (3 * ky + kx) * 8 + c


class PoseNet:
    """The pose-proposal network with its FP32 master parameters and Adam state on the device."""

    def __init__(self, batch: int, device="cuda", params: torch.Tensor | None = None, seed: int = 0):
        L = _abi.lib()
        self.count = int(L.upslam_cnn_param_count())
        self.batch = int(batch)
        self.device = device
        self.ws_bytes = int(L.upslam_cnn_workspace_bytes(self.batch))
        self.ws = torch.zeros(self.ws_bytes, dtype=torch.uint8, device=device)
        self._batches: set = set()  # batch sizes used so far: each has its own error word in ws
        self.params = (params.to(device=device, dtype=torch.float32).clone() if params is not None
                       else self.init_params(seed, device))
        assert self.params.numel() == self.count
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.out = torch.zeros((self.batch, 6), dtype=torch.float32, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.wloss = torch.tensor(LOSS_W, dtype=torch.float32, device=device)

    @staticmethod
    def init_params(seed: int, device) -> torch.Tensor:
        """He-normal conv weights, zero biases, small head (the flat layout of upslam_cnn_*)."""
        g = torch.Generator().manual_seed(seed)
        parts = []
        for l in range(4):
            ci, co = CHANNELS[l], CHANNELS[l + 1]
            parts.append(torch.randn(co * 9 * ci, generator=g, dtype=torch.float64) * math.sqrt(2.0 / (9 * ci)))
            parts.append(torch.zeros(co, dtype=torch.float64))
        parts.append(torch.randn(6 * 128, generator=g, dtype=torch.float64) * math.sqrt(1.0 / 128) * 0.1)
        parts.append(torch.zeros(6, dtype=torch.float64))
        return torch.cat(parts).to(device=device, dtype=torch.float32)

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x: BF16 [B, 64, 256, 8], B <= batch -> FP32 [B, 6] (a view of an internal buffer)."""
        B = x.shape[0]
        assert x.dtype == torch.bfloat16 and x.is_contiguous() and B <= self.batch
        self._batches.add(B)
        _abi.check("upslam_cnn_forward", _abi.lib().upslam_cnn_forward(_p(self.params), _p(x), B, _p(self.out),
                                                                       _p(self.ws), self.ws_bytes, _stream()))
        return self.out[:B]

    def backward(self, x: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
        B = x.shape[0]
        target = target.to(torch.float32).contiguous()
        _abi.check("upslam_cnn_backward",
                   _abi.lib().upslam_cnn_backward(_p(self.params), _p(x), B, _p(self.out), _p(target), _p(self.wloss),
                                                  _p(self.grads), _p(self.loss), _p(self.ws), self.ws_bytes,
                                                  _stream()))
        return self.loss

    def adam(self, lr: float) -> None:
        self.step += 1
        _abi.check("upslam_cnn_adam", _abi.lib().upslam_cnn_adam(_p(self.params), _p(self.grads), _p(self.m),
                                                                 _p(self.v), self.step, float(lr), _stream()))

    def workspace_tensors(self, B: int) -> dict:
        """Views of the tensors the last forward / backward left in the workspace for batch B: BF16 conv
        weights ``wb`` [4], layer outputs ``act`` [4] and pre-activation gradients ``dy`` [4] (NHWC), FP32
        pooled features ``g`` and their gradient ``dg``.  The library holds the first layer's weights in the
        order of its 2x2 space-to-depth convolution ([32][128]); ``wb[0]`` is a copy of them put back in
        the 3x3 order [32][72] (``s2d_feature_source`` gives the correspondence)."""
        L = _abi.lib()
        offs = (ctypes.c_size_t * 16)()
        if L.upslam_cnn_workspace_layout(B, offs) == 0:
            raise ValueError("batch must be positive")

        def view(i, shape, dtype):
            n = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
            return self.ws[offs[i]:offs[i] + n].view(dtype).view(shape)

        out = {"wb": [], "act": [], "dy": []}
        for l in range(4):
            ci, co = CHANNELS[l], CHANNELS[l + 1]
            shape = (B, IN_H >> (l + 1), IN_W >> (l + 1), co)
            if l == 0:
                w_s2d = view(0, (co, S2D_FEATURES), torch.bfloat16)
                w = torch.zeros((co, 9 * ci), dtype=torch.bfloat16, device=w_s2d.device)
                f = [i for i in range(S2D_FEATURES) if s2d_feature_source(i) >= 0]
                w[:, [s2d_feature_source(i) for i in f]] = w_s2d[:, f]
                out["wb"].append(w)
            else:
                out["wb"].append(view(l, (co, 9 * ci), torch.bfloat16))
            out["act"].append(view(4 + l, shape, torch.bfloat16))
            out["dy"].append(view(8 + l, shape, torch.bfloat16))
        out["g"] = view(12, (B, 128), torch.float32)
        out["dg"] = view(13, (B, 128), torch.float32)
        return out

    def check(self) -> None:
        """Raise if a tensor-core wait of any call so far gave up (its outputs were left incomplete)."""
        L = _abi.lib()
        for b in sorted(self._batches):
            off = int(L.upslam_cnn_error_offset(b))
            if int(self.ws[off:off + 4].view(torch.int32).item()) != 0:
                raise RuntimeError(f"pose network: a tensor-core wait gave up (batch {b})")

    def train_step(self, x: torch.Tensor, target: torch.Tensor, lr: float) -> torch.Tensor:
        self.forward(x)
        loss = self.backward(x, target)
        self.adam(lr)
        return loss

    def state_dict(self) -> dict:
        return {"params": self.params.cpu(), "m": self.m.cpu(), "v": self.v.cpu(), "step": self.step}

    def load_state_dict(self, sd: dict) -> None:
        self.params.copy_(sd["params"])
        self.m.copy_(sd["m"])
        self.v.copy_(sd["v"])
        self.step = int(sd["step"])

    def save(self, path: str) -> None:
        """Checkpoint: parameters and Adam state (``torch.save``), so training can resume."""
        torch.save(self.state_dict(), path)

    def load(self, path: str) -> None:
        self.load_state_dict(torch.load(path, map_location="cpu"))


def poses_from_twists(xi: torch.Tensor) -> torch.Tensor:
    """FP64 [B, 12] poses exp(xi^) of FP32 twists [B, 6] (device kernel)."""
    xi = xi.to(torch.float32).contiguous()
    out = torch.empty((xi.shape[0], 12), dtype=torch.float64, device=xi.device)
    _abi.check("upslam_se3_exp", _abi.lib().upslam_se3_exp(_p(xi), xi.shape[0], _p(out), _stream()))
    return out


# ----------------------------------------------------------------------------- pairs from the plain pipeline

class PairBuilder:
    """Keyframe from one sweep (hole fill) + the sweep frame of another, and their 64x256 network input."""

    def __init__(self, sweep_pano, kf_pano, params: Params = Params(), device="cuda"):
        self.params = params
        self.kf = KeyframeBuffer(kf_pano, device)
        self.kf_sweep = SweepFrame(sweep_pano, device)
        self.sw = SweepFrame(sweep_pano, device)
        self.identity = identity_pose(device)
        self._kps = self.kf._ps
        self._sps = self.sw._ps

    def load(self, kf_scan: torch.Tensor, sweep_scan: torch.Tensor) -> None:
        self.kf_sweep.load(kf_scan, self.params)
        self.kf.clear()
        fuse(self.kf, self.kf_sweep, self.identity, self.params, None)
        self.sw.load(sweep_scan, self.params)

    def encode(self, out: torch.Tensor) -> None:
        """Write the BF16 [64, 256, 8] input (keyframe channels 0-3, sweep channels 4-7) into ``out``."""
        L = _abi.lib()
        _abi.check("upslam_downsample", L.upslam_downsample(_p(self.kf.depth), _p(self.kf.nw), self.kf.precision,
                                                            ctypes.byref(self._kps), IN_H, IN_W, DEPTH_SCALE, _p(out),
                                                            IN_C, 0, _stream()))
        _abi.check("upslam_downsample", L.upslam_downsample(_p(self.sw.depth), _p(self.sw.nrm), self.sw.precision,
                                                            ctypes.byref(self._sps), IN_H, IN_W, DEPTH_SCALE, _p(out),
                                                            IN_C, 4, _stream()))


def scene_poses(scene, kind: str, rng: np.random.Generator, n: int, extra=None):
    """n keyframe poses inside a scene (world <- sensor)."""
    import synth
    out = []
    for _ in range(n):
        if kind == "tunnel":
            verts = extra
            i = int(rng.integers(0, len(verts) - 1))
            (x0, y0, h0), (x1, y1, _) = verts[i], verts[i + 1]
            f = rng.uniform(0.1, 0.9)
            x, y = x0 + f * (x1 - x0), y0 + f * (y1 - y0)
            out.append(synth.pose(synth.rot_zyx(math.atan2(y1 - y0, x1 - x0) + rng.uniform(-0.3, 0.3)),
                                  [x, y, 1.0]))
        elif kind == "forest":
            x, y = rng.uniform(-25, 25, size=2)
            out.append(synth.pose(synth.rot_zyx(rng.uniform(-math.pi, math.pi)), [x, y, 1.6 + scene.ground_height(x, y)]))
        else:
            x = rng.uniform(0, 300)
            out.append(synth.pose(synth.rot_zyx(rng.uniform(-0.2, 0.2)), [x, rng.uniform(-2, 2), 1.8]))
    return out


def make_pairs(n_pairs: int, seed: int, device="cuda", keep_scans: bool = False, chunk: int = 256,
               scenes_per_kind: int = 2):
    """n_pairs seeded pairs over tunnel, forest and road scenes -> (x BF16 [n,64,256,8], xi [n,6], extras).

    extras["scans"] (when keep_scans) holds the full-resolution keyframe and sweep scans of every pair."""
    import synth
    from synth import configs
    from synth.gpu import GpuCaster
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device).manual_seed(seed)
    lidar = configs.LIDAR_64
    builder = PairBuilder(lidar.pano(), synth.keyframe_pano(512, 2048, 0.3, 150.0), Params(), device)
    x = torch.zeros((n_pairs, IN_H, IN_W, IN_C), dtype=torch.bfloat16, device=device)
    xi = np.zeros((n_pairs, 6))
    motions = []
    kinds = ["tunnel", "forest", "road"]
    scenes = []
    for k in kinds:
        for s in range(scenes_per_kind):
            sd = seed * 7 + 1000 * kinds.index(k) + s
            if k == "tunnel":
                sc, verts = synth.tunnel_network(sd, length=220.0)
                scenes.append((k, sc, verts))
            elif k == "forest":
                scenes.append((k, synth.forest(sd), None))
            else:
                scenes.append((k, synth.road(sd), None))
    casters = [GpuCaster(sc, lidar, device) for _, sc, _ in scenes]
    scans_kf, scans_sw = [], []
    done = 0
    while done < n_pairs:
        m = min(chunk, n_pairs - done)
        si = int(rng.integers(0, len(scenes)))
        kind, scene, extra = scenes[si]
        kposes = scene_poses(scene, kind, rng, m, extra)
        D = [random_motion(rng) for _ in range(m)]
        sposes = [synth.pose_mul(P, d) for P, d in zip(kposes, D)]
        kscans = casters[si].scans(kposes, gen)
        sscans = casters[si].scans(sposes, gen)
        for i in range(m):
            builder.load(kscans[i], sscans[i])
            builder.encode(x[done + i])
            xi[done + i] = se3_log(D[i])
        if keep_scans:
            scans_kf.append(kscans)
            scans_sw.append(sscans)
        motions.extend(D)
        done += m
    extras = {"motions": motions}
    if keep_scans:
        extras["scans"] = (torch.cat(scans_kf), torch.cat(scans_sw))
    return x, torch.from_numpy(xi).to(device=device, dtype=torch.float32), extras


def train(net: PoseNet, x: torch.Tensor, xi: torch.Tensor, epochs: int = 3, lr: float = 1e-3, seed: int = 0,
          log=None, graph: bool = True) -> list:
    """Mini-batch Adam over (x, xi); the learning rate decays by 10x over the run.  Returns per-epoch mean losses.

    With graph=True the mini-batch gather, forward and backward of a step are captured once as a CUDA graph and
    replayed (the batch indices live in a fixed device buffer); Adam, whose learning rate and bias corrections
    change every step, is launched eagerly after each replay.
    """
    n = x.shape[0]
    B = net.batch
    g = torch.Generator(device=x.device).manual_seed(seed)
    steps = epochs * (n // B)
    idx = torch.zeros(B, dtype=torch.long, device=x.device)
    xb = torch.empty((B,) + tuple(x.shape[1:]), dtype=x.dtype, device=x.device)
    tb = torch.empty((B, 6), dtype=torch.float32, device=x.device)
    xi32 = xi.to(torch.float32).contiguous()

    def body():
        torch.index_select(x, 0, idx, out=xb)
        torch.index_select(xi32, 0, idx, out=tb)
        net.forward(xb)
        net.backward(xb, tb)

    cg = None
    if graph and steps > 0:
        s = torch.cuda.Stream(device=x.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            body()  # first launches (kernel attributes, module loading) outside the capture
            cg = torch.cuda.CUDAGraph()
            with torch.cuda.graph(cg, stream=s):
                body()
        torch.cuda.current_stream().wait_stream(s)
    hist = []
    st = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g, device=x.device)
        tot = torch.zeros((), device=x.device)
        for b in range(n // B):
            idx.copy_(perm[b * B:(b + 1) * B])
            rate = lr * (0.1 ** (st / max(1, steps)))
            if cg is not None:
                cg.replay()
            else:
                body()
            net.adam(rate)
            tot += net.loss[0]
            st += 1
        hist.append(float(tot) / max(1, n // B))
        net.check()
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.5f}")
    return hist


def evaluate(net: PoseNet, x: torch.Tensor, motions: list, scans, params: Params = Params(),
             gate_rms: float = 0.05, gate_quality: float = 0.2, tol_m: float = 0.02, tol_deg: float = 0.1,
             learned_max_iters: int | None = None) -> dict:
    """Plain init + ICP against learned init + ICP (gated, with plain fallback) on held-out pairs.

    Success: final pose within tol_m and tol_deg of the true motion.  The gate accepts the learned start's result
    when ICP reports status OK, inliers / valid >= gate_quality and RMS residual <= gate_rms; otherwise ICP also
    runs from the plain start and the result with the smaller RMS residual is kept.  ``learned_max_iters`` caps
    the Gauss-Newton steps from the learned start (it starts close, so fewer are needed); the plain start and the
    fallback keep ``params.max_iters``.
    """
    import synth
    device = x.device
    n = x.shape[0]
    kf_scans, sw_scans = scans
    sw_pano = _lidar().pano()
    builder = PairBuilder(sw_pano, synth.keyframe_pano(512, 2048, 0.3, 150.0), params, device)
    state = IcpState(builder.kf, device)
    preds = torch.zeros((n, 6), dtype=torch.float32, device=device)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record()
    for b0 in range(0, n, net.batch):
        xb = x[b0:b0 + net.batch].contiguous()
        preds[b0:b0 + xb.shape[0]] = net.forward(xb)
    init_learned = poses_from_twists(preds)
    ev1.record()
    torch.cuda.synchronize()
    t_cnn = time.perf_counter() - t0
    g_cnn = ev0.elapsed_time(ev1) * 1e-3
    ok_plain = ok_learned = ok_gated = fallbacks = 0
    t_plain = t_learned = 0.0
    g_plain = g_learned = 0.0  # device time of the ICP launches (CUDA events), seconds
    I = identity_pose(device)

    import dataclasses
    p_learned = params if learned_max_iters is None else dataclasses.replace(params, max_iters=int(learned_max_iters))

    def run(T0, prm=params):
        """ICP from T0 -> (T, stats, rms, quality, device seconds of the launch)."""
        state.pose.copy_(T0)
        ev0.record()
        icp(builder.kf, builder.sw, state, prm)
        ev1.record()
        st = state.read_stats()
        T = state.pose.cpu().numpy().reshape(3, 4)
        rms = math.sqrt(st["sse"] / max(1, st["inliers"]))
        q = st["inliers"] / max(1, st["valid"])
        return T, st, rms, q, ev0.elapsed_time(ev1) * 1e-3

    iters_plain = iters_learned = 0
    for i in range(n):
        builder.load(kf_scans[i], sw_scans[i])
        truth = motions[i]
        torch.cuda.synchronize()
        a = time.perf_counter()
        Tp, stp, rmsp, qp, gp = run(I)
        torch.cuda.synchronize()
        t_plain += time.perf_counter() - a
        g_plain += gp
        iters_plain += stp["iters"]
        a = time.perf_counter()
        Tl, stl, rmsl, ql, gl = run(init_learned[i], p_learned)
        g_learned += gl
        iters_learned += stl["iters"]
        use = Tl
        if not (stl["status"] == 0 and ql >= gate_quality and rmsl <= gate_rms):
            fallbacks += 1
            Tf, stf, rmsf, qf, gf = run(I)
            g_learned += gf
            iters_learned += stf["iters"]
            if stf["status"] == 0 and (stl["status"] != 0 or rmsf < rmsl):
                use = Tf
        torch.cuda.synchronize()
        t_learned += time.perf_counter() - a
        for T, key in ((Tp, "p"), (Tl, "l"), (use, "g")):
            dt, dr = synth.pose_error(T, truth)
            good = dt <= tol_m and math.degrees(dr) <= tol_deg
            if key == "p":
                ok_plain += good
            elif key == "l":
                ok_learned += good
            else:
                ok_gated += good
    # pairs/s by device time (the ICP launches, and for the gated path also the network's forward over
    # every pair), and by host wall time around the same calls (which adds one stats read per launch)
    return {"pairs": n, "plain_success": ok_plain, "learned_success": ok_learned, "gated_success": ok_gated,
            "fallbacks": fallbacks, "plain_pairs_per_s": n / g_plain, "gated_pairs_per_s": n / (g_learned + g_cnn),
            "plain_pairs_per_s_wall": n / t_plain, "gated_pairs_per_s_wall": n / (t_learned + t_cnn),
            "icp_steps_per_pair_plain": iters_plain / n, "icp_steps_per_pair_gated": iters_learned / n,
            "cnn_ms_per_pair": 1e3 * g_cnn / n}


def _lidar():
    from synth import configs
    return configs.LIDAR_64
