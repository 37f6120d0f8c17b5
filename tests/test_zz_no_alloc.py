"""The allocation-free ICP entry point, called through the C ABI (GPU).

``upslam_icp_noalloc`` is for callers that cannot allocate device memory while
they run: a real-time control loop that must not block on the driver's
allocator, or a plugin whose host runtime owns the device allocator.  Its
workspace is a static array inside the library; the caller passes only inputs
and outputs.  This file is collected last so that a stop-at-first-failure run
has already run every other test.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import synth
from tests.helpers import room_sweep_and_keyframe

torch = pytest.importorskip("torch")
up = pytest.importorskip("paper_2101_00585_gb300")
from paper_2101_00585_gb300 import _abi  # noqa: E402


def _device_inputs():
    c, prm, sp4, sn4, kd, kn = room_sweep_and_keyframe(noise=True)
    kf = up.KeyframeBuffer(c.kf)
    nw = kn.copy()
    nw[..., 3] = (kd > 0).astype(np.float32)
    kf.set(torch.from_numpy(kd).cuda(), torch.from_numpy(nw).cuda())
    sw = up.SweepFrame(c.sweep)
    sw.set(torch.from_numpy(sp4).cuda(), torch.from_numpy(sn4).cuda())
    return kf, sw


@pytest.mark.gpu
def test_noalloc_icp_matches_allocating_icp_on_two_calls():
    """Two calls in a row: the same pose as upslam_icp within the parity tolerance (1e-4 m, 1e-5 rad)."""
    L = up.lib()
    assert L.upslam_icp_noalloc_capacity_bytes() == 561152
    kf, sw = _device_inputs()
    p = up.Params(max_iters=10)
    ref = up.IcpState(kf)
    up.icp(kf, sw, ref, p)
    ref_pose = ref.pose.cpu().numpy().reshape(3, 4)
    ref_rec = ref.read_stats()
    ks, ss, ip = kf.struct(), sw.struct(), p.icp()
    stream = torch.cuda.current_stream().cuda_stream
    # output buffers made up front, so that the second call runs with nothing else allocating
    outs = [(up.identity_pose("cuda"), torch.zeros(_abi.STATS_BYTES, dtype=torch.uint8, device="cuda"))
            for _ in range(2)]
    torch.cuda.synchronize()
    for call, (pose, stats) in enumerate(outs):
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
            reserved_before = torch.cuda.memory_reserved()
        rc = L.upslam_icp_noalloc(ctypes.byref(ks), ctypes.byref(ss), ctypes.c_void_p(pose.data_ptr()),
                                  ctypes.byref(ip), ctypes.c_void_p(stats.data_ptr()), ctypes.c_void_p(stream))
        assert rc == _abi.OK, L.upslam_status_string(rc)
        torch.cuda.synchronize()
        if call == 1:
            # the call after the warm-up one takes no device memory, from the driver or from torch
            assert torch.cuda.mem_get_info()[0] == free_before
            assert torch.cuda.memory_reserved() == reserved_before
        rec = _abi.IcpStats.from_buffer_copy(bytes(stats.cpu().numpy()))
        dt, dr = synth.pose_error(pose.cpu().numpy().reshape(3, 4), ref_pose)
        assert dt < 1e-4 and dr < 1e-5, (call, dt, dr)
        assert rec.status == ref_rec["status"] == 0
        assert rec.iters == ref_rec["iters"]
        assert abs(rec.inliers - ref_rec["inliers"]) <= 2
