"""UPSLAM per-sweep hot path on GB300 (sm_103a): projection, normals, point-to-plane
ICP and keyframe fusion as hand-written CUDA behind the C ABI of include/upslam.h.

    import paper_2101_00585_gb300 as up
    trk = up.Tracker(sweep_pano, keyframe_pano)
    trk.new_keyframe(scan0_cuda)
    trk.track(scan1_cuda)          # pose in trk.state.pose, record in trk.state.stats

The library is built in-tree by ``paper_2101_00585_gb300.build.build()``.
"""
from ._abi import F16, F32, LIB_PATH, UpslamError, lib  # noqa: F401
from .api import (Batch, IcpState, KeyframeBuffer, Params, SweepFrame, Tracker, atrous_normals, empty_zbuf, fuse,  # noqa: F401
                  grid_candidates, grid_score, icp, icp_step, identity_pose, keyframe_consistency, normals, pano_dirs,
                  pano_struct, project, unproject)

__all__ = ["Batch", "Tracker", "Params", "SweepFrame", "KeyframeBuffer", "IcpState", "project", "normals", "atrous_normals", "grid_candidates",
           "grid_score", "keyframe_consistency", "icp",
           "icp_step",
           "fuse", "unproject", "pano_dirs", "pano_struct", "identity_pose", "empty_zbuf", "lib", "UpslamError", "F32",
           "F16", "LIB_PATH"]
