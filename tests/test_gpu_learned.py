"""Learned proposal (workload 5): the BF16 tensor-core network against the FP64 oracle network, the pair
encoding, and what the trained network gains over plain initialisation.

The GPU rounds inputs, conv weights and every activation to BF16 and accumulates in FP32.  The oracle runs in
FP64 on the same BF16-rounded inputs and weights.  Tolerances come from BF16's 2^-9 relative step, compounded
over four layers:
* outputs: relative 3e-2;
* gradients: cosine >= 0.99 and relative norm error <= 0.1 per tensor.

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
    for k in g_ref:
        a, b = g[k].ravel(), g_ref[k].ravel()
        if np.linalg.norm(b) < 1e-12:
            continue
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert cos >= 0.99, (k, cos)
        assert np.linalg.norm(a - b) <= 0.1 * np.linalg.norm(b), k
    net.check()  # no tensor-core wait gave up


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
