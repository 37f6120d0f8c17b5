"""Learned proposal (workload 5): the BF16 tensor-core network against the FP64 oracle network, the pair
encoding, and what the trained network gains over plain initialisation.

The GPU rounds inputs, conv weights and every activation to BF16 and accumulates in FP32.  The oracle runs in
FP64 on the same BF16-rounded inputs and weights.  Tolerances come from BF16's 2^-9 relative step, compounded
over four layers:
* end to end (every layer's rounding compounded): outputs relative 3e-2, gradients cosine >= 0.995 and
  relative norm error <= 8e-2 per tensor (the first layer's weight gradient, four BF16 roundings deep, measured
  6.5 %: its sums cancel, which lifts the 2^-9 rounding of the activations and gradients they multiply to a
  few percent of the sum);
* layer by layer, on the BF16 tensors the GPU held: 4e-3 for what the GPU stores in BF16, 1e-4 for the FP32
  weight and bias gradients (``LAYER_TOL``).

Adam and the SE(3) exponential run in FP32 / FP64 and match to 1e-5 / 1e-12.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import cnn as ocnn
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
up = pytest.importorskip("paper_2101_00585_gb300")
from paper_2101_00585_gb300 import proposal  # noqa: E402


def _bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _flat_params(seed):
    p = ocnn.init_params(seed)
    p["wf"] *= 0.5
    return p


@pytest.mark.parametrize("B", [4, 3, 1, 40])
def test_forward_backward_match_oracle(B):
    """B = 3 leaves ragged tensor-core tiles (the last layer's 192 rows are 1.5 tiles of 128); B = 1 gives the
    last layer a single half-empty tile and each weight gradient one K slice; B = 40 gives the first layer 1280
    output tiles, so every persistent CTA runs several tiles through one load pipeline.  The bias gradients
    come out of the weight-gradient GEMM (an appended feature of ones) and are checked with the rest."""
    rng = np.random.default_rng(5 + B)
    x = rng.uniform(-1, 1, size=(B, 64, 256, 8)) * (rng.random((B, 64, 256, 1)) < 0.7)
    xb = _bf16(x)
    p = _flat_params(6)
    flat = ocnn.flatten(p)
    net = proposal.PoseNet(B, params=torch.from_numpy(flat))
    x_dev = torch.from_numpy(xb.astype(np.float32)).to(torch.bfloat16).cuda().contiguous()
    out = net.forward(x_dev).cpu().numpy().astype(np.float64)
    # the oracle on the BF16-rounded input and conv weights (the GPU's operands)
    pr = {k: (_bf16(v) if k.startswith("w") and k != "wf" else v) for k, v in p.items()}
    ref, cache = ocnn.forward(pr, xb)
    assert np.linalg.norm(out - ref) <= 3e-2 * np.linalg.norm(ref)
    target = rng.standard_normal((B, 6)) * 0.3
    wts = np.array(proposal.LOSS_W)
    L_ref, dout = ocnn.loss(ref, target, wts)
    g_ref = ocnn.backward(pr, cache, dout)
    loss = net.backward(x_dev, torch.from_numpy(target).cuda())
    assert abs(float(loss) - L_ref) <= 3e-2 * abs(L_ref)
    g = ocnn.unflatten(net.grads.cpu().numpy().astype(np.float64))
    worst = {}
    for k in g_ref:
        a, b = g[k].ravel(), g_ref[k].ravel()
        if np.linalg.norm(b) < 1e-12:
            continue
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        worst[k] = (cos, float(np.linalg.norm(a - b) / np.linalg.norm(b)))
        assert cos >= 0.995, (k, cos)
        assert np.linalg.norm(a - b) <= 8e-2 * np.linalg.norm(b), (k, worst[k])
    net.check()  # no tensor-core wait gave up


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


def _f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def _layer_errors(net, x_dev, B, target, onet=ocnn):
    """Each layer of the GPU's forward and backward against the oracle's arithmetic for that layer alone,
    fed the GPU's own BF16 tensors (its input, its weights, the gradient arriving from above), so the
    BF16 rounding of earlier layers does not enter.  -> {check name: relative Frobenius error}."""
    ws = net.workspace_tensors(B)
    wb = [_f64(w) for w in ws["wb"]]
    act = [_f64(a) for a in ws["act"]]
    dy = [_f64(d) for d in ws["dy"]]
    ins = [_f64(x_dev)] + act[:3]
    p = ocnn.unflatten(net.params.cpu().numpy().astype(np.float64))
    g = ocnn.unflatten(net.grads.cpu().numpy().astype(np.float64))
    err = {}
    for l in range(4):
        co = ocnn.CHANNELS[l + 1]
        cols = onet.im2col(ins[l])
        pre = cols @ wb[l].T + p[f"b{l}"]
        err[f"act{l}"] = _rel(act[l].reshape(-1, co), np.maximum(pre, 0.0))
        dyl = dy[l].reshape(-1, co)
        err[f"w{l}"] = _rel(g[f"w{l}"].reshape(co, -1), dyl.T @ cols)
        err[f"b{l}"] = _rel(g[f"b{l}"], dyl.sum(axis=0))
        if l > 0:
            dx = onet.col2im(dyl @ wb[l], ins[l].shape) * (act[l - 1] > 0)
            err[f"dx{l}"] = _rel(dy[l - 1], dx)
    # the head: pooled features, the output, and the gradient it sends into the last feature map
    gpool = act[3].mean(axis=(1, 2))
    out = gpool @ p["wf"].T + p["bf"]
    err["pool"] = _rel(_f64(ws["g"]), gpool)
    err["out"] = _rel(net.out[:B].cpu().numpy().astype(np.float64), out)
    _, dout = ocnn.loss(out, target, np.array(proposal.LOSS_W))
    H, W = act[3].shape[1:3]
    da = np.broadcast_to((dout @ p["wf"])[:, None, None, :] / (H * W), act[3].shape) * (act[3] > 0)
    err["dy3"] = _rel(dy[3], da)
    err["wf"] = _rel(g["wf"], dout.T @ gpool)
    err["bf"] = _rel(g["bf"], dout.sum(axis=0))
    return err


# Tolerances per check, from the arithmetic: values the GPU stores in BF16 (layer outputs, the gradients
# passed down) carry its 2^-9 relative rounding, plus FP32 accumulation; weight and bias gradients are FP32
# sums of exact BF16 x BF16 products (2^-24 per addition over reductions of up to 1.6e5 terms, in slices)
LAYER_TOL = {"act": 4e-3, "dx": 4e-3, "dy": 4e-3, "w": 1e-4, "b": 1e-4, "pool": 1e-5, "out": 1e-5, "wf": 1e-5,
             "bf": 1e-5}


def _tol(name):
    return LAYER_TOL[name.rstrip("0123456789")]


def _run_layers(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(B, 64, 256, 8)) * (rng.random((B, 64, 256, 1)) < 0.7)
    net = proposal.PoseNet(B, params=torch.from_numpy(ocnn.flatten(_flat_params(seed + 1))))
    x_dev = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).cuda().contiguous()
    net.forward(x_dev)
    target = rng.standard_normal((B, 6)) * 0.3
    net.backward(x_dev, torch.from_numpy(target).cuda())
    torch.cuda.synchronize()
    net.check()
    return net, x_dev, target


@pytest.mark.parametrize("B", [3, 24])
def test_every_layer_matches_oracle_on_the_gpus_own_tensors(B):
    """Layer by layer: forward outputs, weight and bias gradients, and the gradient passed to the layer below
    (the data-gradient GEMM with its tap parity classes and ReLU mask), each against the oracle's FP64
    arithmetic of that one layer on the BF16 tensors the GPU held."""
    net, x_dev, target = _run_layers(B, 40 + B)
    err = _layer_errors(net, x_dev, B, target)
    bad = {k: v for k, v in err.items() if not v <= _tol(k)}
    assert not bad, (bad, err)


def test_layer_check_catches_a_dropped_tap_in_the_data_gradient(monkeypatch):
    """The per-layer check has the power to see a one-tap mistake: with one of the nine taps dropped from
    the oracle's col2im (the adjoint the data gradient is checked against), the dx checks fail."""
    B = 3
    net, x_dev, target = _run_layers(B, 43)

    class Dropped:
        im2col = staticmethod(ocnn.im2col)

        @staticmethod
        def col2im(dcols, shape):
            Bn, H, W, C = shape
            d = dcols.reshape(Bn, H // 2, W // 2, 3, 3, C).copy()
            d[:, :, :, 2, 1, :] = 0.0  # the tap (ky, kx) = (2, 1) forgotten
            return ocnn.col2im(d.reshape(dcols.shape), shape)

    err = _layer_errors(net, x_dev, B, target, onet=Dropped)
    assert all(err[f"dx{l}"] > 10 * _tol("dx") for l in (1, 2, 3)), err


def test_adam_matches_oracle():
    flat = ocnn.flatten(_flat_params(7))
    rng = np.random.default_rng(8)
    net = proposal.PoseNet(2, params=torch.from_numpy(flat))
    grads = rng.standard_normal(flat.size) * 1e-2
    net.grads.copy_(torch.from_numpy(grads))
    p, m, v = ocnn.unflatten(flat.copy()), ocnn.unflatten(np.zeros_like(flat)), ocnn.unflatten(np.zeros_like(flat))
    gd = ocnn.unflatten(grads)
    for t in (1, 2, 3):
        net.adam(1e-3)
        ocnn.adam_step(p, gd, m, v, t, lr=1e-3)
    got = net.params.cpu().numpy().astype(np.float64)
    want = ocnn.flatten(p)
    assert np.allclose(got, want, rtol=1e-5, atol=1e-7)


def test_se3_exp_batch_matches_oracle():
    rng = np.random.default_rng(9)
    xi = (rng.standard_normal((64, 6)) * np.array([0.3, 0.3, 0.3, 1, 1, 1])).astype(np.float32)
    got = proposal.poses_from_twists(torch.from_numpy(xi).cuda()).cpu().numpy().reshape(-1, 3, 4)
    I = np.hstack([np.eye(3), np.zeros((3, 1))])
    for i in range(64):
        want = oracle.se3_exp_left(xi[i].astype(np.float64), I)
        assert np.allclose(got[i], want, atol=1e-12)
        # and the host log inverts it
        assert np.allclose(proposal.se3_log(want), xi[i], atol=1e-6)


def test_downsample_matches_reference():
    kp = synth.keyframe_pano(512, 2048)
    rng = np.random.default_rng(10)
    depth = np.where(rng.random((512, 2048)) < 0.1, rng.uniform(1, 50, (512, 2048)), 0).astype(np.float32)
    nrm = np.zeros((512, 2048, 4), np.float32)
    v = rng.standard_normal((512, 2048, 3))
    nrm[..., :3] = v / np.linalg.norm(v, axis=-1, keepdims=True)
    nrm[..., 3] = (depth > 0).astype(np.float32)
    kf = up.KeyframeBuffer(kp)
    kf.set(torch.from_numpy(depth).cuda(), torch.from_numpy(nrm).cuda())
    out = torch.zeros((64, 256, 8), dtype=torch.bfloat16, device="cuda")
    import ctypes
    from paper_2101_00585_gb300 import _abi
    ps = up.pano_struct(kp)
    rc = up.lib().upslam_downsample(ctypes.c_void_p(kf.depth.data_ptr()), ctypes.c_void_p(kf.nw.data_ptr()), 0,
                                    ctypes.byref(ps), 64, 256, 20.0, ctypes.c_void_p(out.data_ptr()), 8, 4,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _abi.OK
    got = out.float().cpu().numpy()
    want = ocnn.downsample(depth, nrm, 64, 256, 20.0)
    assert np.allclose(got[..., 4:], want, atol=2 ** -8 * np.maximum(1, np.abs(want)) + 1e-3)
    assert np.all(got[..., :4] == 0)


def test_learned_proposal_gains_over_plain_init():
    """Trained on pairs the plain pipeline makes, the gated learned start registers more held-out large-motion
    pairs within 2 cm / 0.1 deg than ICP from the plain (zero-velocity) start."""
    torch.manual_seed(0)
    x, xi, _ = proposal.make_pairs(32768, seed=11)
    net = proposal.PoseNet(128)
    hist = proposal.train(net, x, xi, epochs=8, lr=2e-3, seed=12)
    assert hist[-1] < hist[0]
    xt, xit, ext = proposal.make_pairs(256, seed=13, keep_scans=True)
    res = proposal.evaluate(net, xt, ext["motions"], ext["scans"])
    print("\nlearned proposal:", res, "train loss", [round(h, 4) for h in hist])
    assert res["gated_success"] > res["plain_success"]


def test_train_graph_replay_matches_eager():
    """The captured step (gather, forward, backward replayed as one CUDA graph, Adam eager) trains like the eager
    step.  The weight gradients are FP32 atomic sums, whose order varies, so the runs agree to rounding."""
    rng = np.random.default_rng(21)
    n, B = 384, 64
    x = torch.from_numpy((rng.uniform(-1, 1, (n, 64, 256, 8)) * (rng.random((n, 64, 256, 1)) < 0.7))
                         .astype(np.float32)).to(torch.bfloat16).cuda()
    xi = torch.from_numpy(rng.standard_normal((n, 6)) * 0.3).cuda()
    flat = torch.from_numpy(ocnn.flatten(_flat_params(22)))
    nets, hists = [], []
    for graph in (False, True):
        net = proposal.PoseNet(B, params=flat)
        hists.append(proposal.train(net, x, xi, epochs=2, lr=2e-3, seed=23, graph=graph))
        nets.append(net)
    assert np.allclose(hists[0], hists[1], rtol=1e-3), hists
    a, b = nets[0].params.cpu().numpy(), nets[1].params.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(a)
    assert nets[1].step == 2 * (n // B)
