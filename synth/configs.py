"""The five seeded synthetic workloads (scene, sensor, keyframe geometry, motion).

Seeds are 20210101 + workload number; every scan draws its noise from its own
``numpy.random.default_rng((seed, scan_index))`` stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import (Lidar, Pano, Scene, box_room, campus, forest, keyframe_pano, line_trajectory, perturb, pose,
               relative, rot_zyx, road, scan, tunnel_network, tunnel_trajectory)

SEED0 = 20210101


def seed(cfg: int) -> int:
    return SEED0 + cfg


def scan_rng(cfg: int, k: int) -> np.random.Generator:
    return np.random.default_rng((seed(cfg), k))


# ----------------------------------------------------------------------------- 1: box room, single registration

LIDAR_16 = Lidar(beams=16, cols=512, fov_top_deg=15.0, fov_bot_deg=-15.0, r_min=0.3, r_max=30.0, sigma=0.01,
                 dropout=0.02)


@dataclass
class RoomCase:
    scene: Scene
    lidar: Lidar
    sweep: Pano
    kf: Pano
    P_w_kf: np.ndarray
    P_w_s: np.ndarray
    T_true: np.ndarray  # keyframe <- sweep
    scan: np.ndarray


def room_case(noise: bool = True, trans_m: float = 0.05, rot_deg: float = 2.0, cfg_seed: int | None = None,
              kf_rows: int = 256, kf_cols: int = 512) -> RoomCase:
    """16 x 512 sweep in the 10 x 8 x 3 m room vs a 256 x 512 keyframe from a second pose."""
    s = seed(1) if cfg_seed is None else cfg_seed
    rng = np.random.default_rng(s)
    scene = box_room(s)
    P_w_kf = pose(rot_zyx(rng.uniform(-math.pi, math.pi), 0.0, 0.0), [0.4, -0.3, 1.3])
    P_w_s = perturb(P_w_kf, rng, trans_m, math.radians(rot_deg))
    lidar = LIDAR_16 if noise else Lidar(**{**LIDAR_16.__dict__, "sigma": 0.0, "dropout": 0.0})
    sc = scan(scene, lidar, P_w_s, np.random.default_rng((s, 1)))
    return RoomCase(scene, lidar, lidar.pano(), keyframe_pano(kf_rows, kf_cols, 0.3, 30.0), P_w_kf, P_w_s,
                    relative(P_w_kf, P_w_s), sc)


# ----------------------------------------------------------------------------- 2: tunnel sequence (headline)

LIDAR_64 = Lidar(beams=64, cols=1024, fov_top_deg=16.6, fov_bot_deg=-16.6, r_min=0.5, r_max=120.0, sigma=0.02,
                 dropout=0.02)


@dataclass
class Sequence:
    scene: Scene
    lidar: Lidar
    sweep: Pano
    kf: Pano
    poses: list            # world <- sensor, ground truth
    kf_every: int          # a new keyframe every kf_every scans
    cfg: int

    def scan(self, k: int) -> np.ndarray:
        return scan(self.scene, self.lidar, self.poses[k], scan_rng(self.cfg, k))

    def scans(self, k0: int, n: int) -> np.ndarray:
        return np.stack([self.scan(k) for k in range(k0, k0 + n)])


def tunnel_sequence(n_scans: int = 2000, step: float = 0.1, kf_rows: int = 512, kf_cols: int = 2048,
                    lidar: Lidar = LIDAR_64) -> Sequence:
    """64 x 1024 sweeps every 0.1 m along a 200 m corridor network; 512 x 2048 keyframes every 5 m."""
    rng = np.random.default_rng(seed(2))
    scene, verts = tunnel_network(seed(2), length=n_scans * step + 30.0)
    poses = tunnel_trajectory(verts, n_scans, step, rng)
    return Sequence(scene, lidar, lidar.pano(), keyframe_pano(kf_rows, kf_cols, 0.3, 150.0), poses,
                    max(1, int(round(5.0 / step))), 2)


# ----------------------------------------------------------------------------- 3: campus, precision form

LIDAR_128 = Lidar(beams=128, cols=2048, fov_top_deg=22.5, fov_bot_deg=-22.5, r_min=0.5, r_max=120.0, sigma=0.02,
                  dropout=0.02)


def campus_sequence(n_scans: int = 1000, step: float = 0.5) -> Sequence:
    """128 x 2048 sweeps every 0.5 m over 500 m of campus; 1024 x 4096 keyframes every 5 m."""
    rng = np.random.default_rng(seed(3))
    scene = campus(seed(3))
    poses = line_trajectory(n_scans, step, rng, y0=0.0, height=1.8, scene=scene, heading=0.0)
    return Sequence(scene, LIDAR_128, LIDAR_128.pano(), keyframe_pano(1024, 4096, 0.3, 150.0), poses,
                    max(1, int(round(5.0 / step))), 3)


# ----------------------------------------------------------------------------- 4: forest, batched problems

KF_SIZES_4 = ((256, 1024),) * 22 + ((512, 2048),) * 21 + ((1024, 4096),) * 21


@dataclass
class BatchCase:
    scene: Scene
    lidar: Lidar
    sweep: Pano
    scan: np.ndarray
    P_w_s: np.ndarray
    kf_panos: list
    kf_poses: list          # world <- keyframe
    T_true: list            # keyframe <- sweep, per keyframe
    T_init: list            # [n_kf][n_hyp] initial hypotheses
    n_hyp: int


def forest_batch(n_kf: int = 64, n_hyp: int = 8, max_trans: float = 2.0, max_rot_deg: float = 20.0,
                 kf_sizes=KF_SIZES_4) -> BatchCase:
    """One 64 x 1024 forest sweep vs n_kf nearby keyframes of mixed sizes, n_hyp seeded hypotheses each."""
    rng = np.random.default_rng(seed(4))
    scene = forest(seed(4))
    lid = LIDAR_64
    P_w_s = pose(rot_zyx(rng.uniform(-math.pi, math.pi), 0.0, 0.0), [0.0, 0.0, 1.6 + scene.ground_height(0, 0)])
    sc = scan(scene, lid, P_w_s, scan_rng(4, 0))
    panos, kposes, Tt, Ti = [], [], [], []
    for i in range(n_kf):
        rows, cols = kf_sizes[i % len(kf_sizes)]
        panos.append(keyframe_pano(rows, cols, 0.3, 150.0))
        ang = rng.uniform(0, 2 * math.pi)
        dist = rng.uniform(0.5, 4.0)
        x, y = dist * math.cos(ang), dist * math.sin(ang)
        Pk = pose(rot_zyx(rng.uniform(-math.pi, math.pi), 0.0, 0.0), [x, y, 1.6 + scene.ground_height(x, y)])
        kposes.append(Pk)
        T = relative(Pk, P_w_s)
        Tt.append(T)
        hyps = []
        for h in range(n_hyp):
            tm = max_trans * rng.uniform(0.0, 1.0)
            rr = math.radians(max_rot_deg) * rng.uniform(0.0, 1.0)
            hyps.append(perturb(T, rng, tm, rr))
        Ti.append(hyps)
    return BatchCase(scene, lid, lid.pano(), sc, P_w_s, panos, kposes, Tt, Ti, n_hyp)


# ----------------------------------------------------------------------------- 5: learned proposal pairs

def pair_scenes(cfg_seed: int):
    return [tunnel_network(cfg_seed)[0], forest(cfg_seed + 1), road(cfg_seed + 2)]
