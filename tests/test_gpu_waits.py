"""Bounded device waits end in a status, not a hang (GPU).

Every wait in the persistent kernels has a limit: a grid-barrier wait of the
ICP launch gives up after a clock-cycle budget and records UPSLAM_ERR_TIMEOUT,
and an mbarrier wait of the tensor-core GEMMs gives up after a global-timer
budget, drains what its CTA issued, frees its tensor memory and sets the
network's error word.  The test entry points below shorten the limit to about
a millisecond and withhold one signal, so the wait cannot end; the tests check
the reported status and that the device keeps working afterwards.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from tests.helpers import IDENTITY, room_sweep_and_keyframe

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
up = pytest.importorskip("paper_2101_00585_gb300")
from paper_2101_00585_gb300 import _abi  # noqa: E402


def _room_buffers():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf = up.KeyframeBuffer(c.kf)
    nw = kn.copy()
    nw[..., 3] = (kd > 0).astype(np.float32)
    kf.set(torch.from_numpy(kd).cuda(), torch.from_numpy(nw).cuda())
    sw = up.SweepFrame(c.sweep)
    sw.set(torch.from_numpy(sp4).cuda(), torch.from_numpy(sn4).cuda())
    return kf, sw


def test_icp_grid_barrier_wait_gives_up_with_timeout_status():
    L = up.lib()
    kf, sw = _room_buffers()
    p = up.Params(max_iters=10)
    ref = up.IcpState(kf)
    up.icp(kf, sw, ref, p)
    probe = up.IcpState(kf)
    ks, ss, ip = kf.struct(), sw.struct(), p.icp()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.upslam_icp_wait_probe(ctypes.byref(ks), ctypes.byref(ss), ctypes.c_void_p(probe.pose.data_ptr()),
                                 ctypes.byref(ip), ctypes.c_void_p(probe.stats.data_ptr()),
                                 ctypes.c_void_p(probe.ws.data_ptr()), probe.ws_bytes, ctypes.c_longlong(2_000_000),
                                 stream)
    assert rc == _abi.OK
    torch.cuda.synchronize()
    rec = probe.read_stats()
    assert rec["status"] == _abi.ERR_TIMEOUT
    assert np.array_equal(probe.pose.cpu().numpy().reshape(3, 4), IDENTITY)
    # a limit outside 1000 .. 4e9 cycles is refused before any launch
    assert L.upslam_icp_wait_probe(ctypes.byref(ks), ctypes.byref(ss), ctypes.c_void_p(probe.pose.data_ptr()),
                                   ctypes.byref(ip), ctypes.c_void_p(probe.stats.data_ptr()),
                                   ctypes.c_void_p(probe.ws.data_ptr()), probe.ws_bytes, ctypes.c_longlong(10),
                                   stream) == _abi.ERR_INVALID_ARG
    # the device keeps working: with the workspace zeroed again the same state registers as before
    probe.ws.zero_()
    probe.pose.copy_(up.identity_pose("cuda"))
    up.icp(kf, sw, probe, p)
    torch.cuda.synchronize()
    assert torch.equal(probe.pose, ref.pose)
    assert probe.read_stats()["status"] == 0


def test_cnn_tensor_core_wait_gives_up_and_sets_the_error_word():
    from paper_2101_00585_gb300 import proposal
    L = up.lib()
    B = 64
    net = proposal.PoseNet(B, seed=3)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand((B, proposal.IN_H, proposal.IN_W, proposal.IN_C), generator=g, device="cuda").to(torch.bfloat16)
    ref = net.forward(x).clone()
    torch.cuda.synchronize()
    off = int(L.upslam_cnn_error_offset(B))
    word = net.ws[off:off + 4].view(torch.int32)
    assert int(word.item()) == 0
    out = torch.zeros((B, 6), dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.upslam_cnn_forward_wait_probe(ctypes.c_void_p(net.params.data_ptr()), ctypes.c_void_p(x.data_ptr()), B,
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(net.ws.data_ptr()),
                                         net.ws_bytes, ctypes.c_ulonglong(1_000_000), stream)
    assert rc == _abi.OK
    torch.cuda.synchronize()
    assert int(word.item()) != 0
    with pytest.raises(RuntimeError):
        net.check()
    assert L.upslam_cnn_forward_wait_probe(ctypes.c_void_p(net.params.data_ptr()), ctypes.c_void_p(x.data_ptr()), B,
                                           ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(net.ws.data_ptr()),
                                           net.ws_bytes, ctypes.c_ulonglong(10), stream) == _abi.ERR_INVALID_ARG
    # the device keeps working: with the word cleared the forward pass gives the same outputs again
    word.zero_()
    again = net.forward(x).clone()
    torch.cuda.synchronize()
    assert torch.equal(again, ref)
    assert int(word.item()) == 0
