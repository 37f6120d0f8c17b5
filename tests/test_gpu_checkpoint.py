"""Checkpoint and resume (GPU): a keyframe and the pose network's training state survive a round trip to disk,
and training resumed from a checkpoint continues exactly as the uninterrupted run."""
from __future__ import annotations

import numpy as np
import pytest

from synth import configs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
up = pytest.importorskip("paper_2101_00585_gb300")


@pytest.mark.parametrize("precision", [0, 1])
def test_keyframe_round_trip(tmp_path, precision):
    seq = configs.tunnel_sequence(n_scans=3)
    trk = up.Tracker(seq.sweep, seq.kf, up.Params(accept_quality=0.1), precision=precision)
    trk.new_keyframe(torch.from_numpy(seq.scan(0)).cuda())
    trk.track(torch.from_numpy(seq.scan(1)).cuda())
    path = str(tmp_path / "kf.npz")
    trk.kf.save(path)
    kf = up.KeyframeBuffer.load(path)
    assert kf.precision == precision and (int(kf.pp.rows), int(kf.pp.cols)) == (int(seq.kf.rows), int(seq.kf.cols))
    assert torch.equal(kf.depth, trk.kf.depth) and torch.equal(kf.nw, trk.kf.nw)
    assert torch.equal(kf.dirs, trk.kf.dirs)


def test_training_resumes_from_a_checkpoint(tmp_path):
    from paper_2101_00585_gb300 import proposal
    B = 8
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.rand((B, proposal.IN_H, proposal.IN_W, proposal.IN_C), generator=g, device="cuda").to(torch.bfloat16)
    t = torch.rand((B, 6), generator=g, device="cuda") * 0.2
    a = proposal.PoseNet(B, seed=4)
    for _ in range(2):
        a.train_step(x, t, 1e-3)
    path = str(tmp_path / "net.pt")
    a.save(path)
    b = proposal.PoseNet(B, seed=9)
    b.load(path)
    assert torch.equal(a.params, b.params) and torch.equal(a.m, b.m) and torch.equal(a.v, b.v) and a.step == b.step
    # the next step from the checkpoint: same parameters within FP32 gradient summation order
    a.train_step(x, t, 1e-3)
    b.train_step(x, t, 1e-3)
    torch.cuda.synchronize()
    assert np.allclose(a.params.cpu().numpy(), b.params.cpu().numpy(), rtol=1e-5, atol=1e-6)
