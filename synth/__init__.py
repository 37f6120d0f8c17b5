"""Seeded synthetic spinning-lidar inputs (scenes, sensors, trajectories, scans).

This module generates inputs only.  It holds none of the registration or fusion
arithmetic of the method, so the CPU oracle (``oracle/``) and the CUDA library
can both consume what it produces without sharing code with each other.

Conventions
-----------
* World frame: z up.  Sensor frame: x forward, y left, z up.
* A pose is a 3x4 FP64 array ``[R | t]`` mapping sensor coordinates to world
  coordinates (or, for a relative pose, sweep to keyframe).
* Panorama geometry (paper Sec. III, panoramic depth images; keyframes may be
  wider than the sensor's vertical field of view): row 0 is the top edge at
  elevation ``el_top``; column 0 starts at azimuth +pi and columns advance
  clockwise.  ``s_az = cols / 2pi`` and ``s_el = rows / (el_top - el_bot)``
  are computed in FP64 and rounded once to FP32; those FP32 values are the
  panorama's definition from then on.
* A scan is an ``(N, 4)`` FP32 array ``(x, y, z, valid)`` in sensor
  coordinates, ordered column-major like a spinning sensor emits it:
  point ``i = col * beams + beam``.  Invalid points (no return, dropout) have
  ``valid = 0`` and ``xyz = 0``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_raycast.so")
PRIM_STRIDE = 16
PLANE, OBB, ROOM, VCYL, ARCH, HFIELD = range(6)

_lib = None


def build(force: bool = False) -> str:
    """Compile the ray caster with gcc (OpenMP over rays)."""
    src = os.path.join(_HERE, "raycast.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", src, "-o", _SO, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.synth_cast.argtypes = [dp, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_double, dp, dp,
                                   ctypes.POINTER(ctypes.c_int32)]
        lib.synth_cast.restype = ctypes.c_int
        lib.synth_hfield_height.argtypes = [dp, ctypes.c_double, ctypes.c_double]
        lib.synth_hfield_height.restype = ctypes.c_double
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------- geometry helpers

def rot_zyx(yaw: float, pitch: float = 0.0, roll: float = 0.0) -> np.ndarray:
    """R = Rz(yaw) Ry(pitch) Rx(roll), FP64."""
    cy, sy, cp, sp, cr, sr = (math.cos(yaw), math.sin(yaw), math.cos(pitch), math.sin(pitch),
                              math.cos(roll), math.sin(roll))
    rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1.0]])
    ry = np.array([[cp, 0, sp], [0, 1.0, 0], [-sp, 0, cp]])
    rx = np.array([[1.0, 0, 0], [0, cr, -sr], [0, sr, cr]])
    return rz @ ry @ rx


def rot_axis_angle(axis, angle: float) -> np.ndarray:
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    k = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * k + (1 - math.cos(angle)) * (k @ k)


def pose(R: np.ndarray, t) -> np.ndarray:
    P = np.zeros((3, 4))
    P[:, :3] = R
    P[:, 3] = t
    return P


def pose_inv(P: np.ndarray) -> np.ndarray:
    R, t = P[:, :3], P[:, 3]
    return pose(R.T, -R.T @ t)


def pose_mul(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    return pose(A[:, :3] @ B[:, :3], A[:, :3] @ B[:, 3] + A[:, 3])


def relative(P_w_kf: np.ndarray, P_w_s: np.ndarray) -> np.ndarray:
    """Keyframe-from-sweep pose T = P_w_kf^-1 P_w_s."""
    return pose_mul(pose_inv(P_w_kf), P_w_s)


def pose_error(A: np.ndarray, B: np.ndarray):
    """(translation error m, rotation error rad) between two poses.

    The angle of R_A^T R_B is atan2(|vee(M - M^T)| / 2, (tr M - 1) / 2), which stays
    accurate for tiny angles (an arccos of the trace would not)."""
    dt = float(np.linalg.norm(A[:, 3] - B[:, 3]))
    M = A[:, :3].T @ B[:, :3]
    s = 0.5 * math.sqrt((M[2, 1] - M[1, 2]) ** 2 + (M[0, 2] - M[2, 0]) ** 2 + (M[1, 0] - M[0, 1]) ** 2)
    c = 0.5 * (np.trace(M) - 1.0)
    return dt, float(math.atan2(s, c))


def perturb(P: np.ndarray, rng: np.random.Generator, trans_m: float, rot_rad: float) -> np.ndarray:
    """P D for a random rigid motion D of exactly (trans_m, rot_rad), so that P^-1 (P D) = D."""
    ax = rng.standard_normal(3)
    dv = rng.standard_normal(3)
    dv = dv / np.linalg.norm(dv) * trans_m
    D = pose(rot_axis_angle(ax, rot_rad), dv)
    return pose_mul(P, D)


# ----------------------------------------------------------------------------- panorama / lidar

@dataclass(frozen=True)
class Pano:
    """Panorama geometry; the FP32 fields are the definition used by both sides."""
    rows: int
    cols: int
    el_top: np.float32
    s_az: np.float32
    s_el: np.float32
    r_min: np.float32
    r_max: np.float32
    el_top64: float = 0.0
    el_bot64: float = 0.0

    @staticmethod
    def make(rows: int, cols: int, el_top: float, el_bot: float, r_min: float, r_max: float) -> "Pano":
        return Pano(rows, cols, np.float32(el_top), np.float32(cols / (2.0 * math.pi)),
                    np.float32(rows / (el_top - el_bot)), np.float32(r_min), np.float32(r_max),
                    float(el_top), float(el_bot))

    @property
    def pixels(self) -> int:
        return self.rows * self.cols

    def pixel_dirs(self) -> np.ndarray:
        """FP64 unit directions through the pixel centres, shape (rows, cols, 3)."""
        v = np.arange(self.rows) + 0.5
        u = np.arange(self.cols) + 0.5
        el = float(self.el_top) - v / float(self.s_el)
        az = math.pi - u / float(self.s_az)
        ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
        return np.stack([ce * np.cos(az)[None, :], ce * np.sin(az)[None, :],
                         np.broadcast_to(se, (self.rows, self.cols))], axis=-1)


def keyframe_pano(rows: int, cols: int, r_min: float = 0.3, r_max: float = 150.0,
                  half_fov_deg: float = 45.0) -> Pano:
    """Keyframe panoramas span +-45 deg vertically, wider than the sensor."""
    h = math.radians(half_fov_deg)
    return Pano.make(rows, cols, h, -h, r_min, r_max)


@dataclass(frozen=True)
class Lidar:
    beams: int
    cols: int
    fov_top_deg: float
    fov_bot_deg: float
    r_min: float
    r_max: float
    sigma: float
    dropout: float

    @property
    def n_points(self) -> int:
        return self.beams * self.cols

    def pano(self) -> Pano:
        """Sweep panorama: one row per beam; rows extend half a beam spacing past the FOV."""
        top, bot = math.radians(self.fov_top_deg), math.radians(self.fov_bot_deg)
        half = 0.5 * (top - bot) / (self.beams - 1)
        return Pano.make(self.beams, self.cols, top + half, bot - half, self.r_min, self.r_max)

    def directions(self) -> np.ndarray:
        """Sensor-frame unit ray directions, column-major, shape (N, 3), FP64."""
        top, bot = math.radians(self.fov_top_deg), math.radians(self.fov_bot_deg)
        el = top - (top - bot) * np.arange(self.beams) / (self.beams - 1)
        az = math.pi - (np.arange(self.cols) + 0.5) * (2.0 * math.pi / self.cols)
        E = np.broadcast_to(el[None, :], (self.cols, self.beams)).reshape(-1)
        A = np.broadcast_to(az[:, None], (self.cols, self.beams)).reshape(-1)
        return np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], axis=-1)


# ----------------------------------------------------------------------------- scenes

@dataclass
class Scene:
    prims: np.ndarray = field(default_factory=lambda: np.zeros((0, PRIM_STRIDE)))
    name: str = ""

    def add(self, kind: int, *params: float) -> None:
        row = np.zeros(PRIM_STRIDE)
        row[0] = kind
        row[1:1 + len(params)] = params
        self.prims = np.vstack([self.prims, row[None, :]])

    def cast(self, origin, dirs_world: np.ndarray, tmax: float):
        lib = _load()
        dirs = np.ascontiguousarray(dirs_world, dtype=np.float64)
        n = dirs.shape[0]
        prims = np.ascontiguousarray(self.prims, dtype=np.float64)
        o = np.ascontiguousarray(origin, dtype=np.float64)
        t = np.empty(n)
        nrm = np.empty((n, 3))
        ids = np.empty(n, dtype=np.int32)
        lib.synth_cast(_dptr(prims), prims.shape[0], _dptr(o), _dptr(dirs), n, float(tmax), _dptr(t),
                       _dptr(nrm), ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return t, nrm, ids

    def ground_height(self, x: float, y: float) -> float:
        lib = _load()
        for row in self.prims:
            if int(row[0]) == HFIELD:
                r = np.ascontiguousarray(row)
                return lib.synth_hfield_height(_dptr(r), x, y)
        return 0.0


def box_room(seed: int) -> Scene:
    """10 x 8 x 3 m room with two box obstacles."""
    rng = np.random.default_rng(seed)
    s = Scene(name="box_room")
    s.add(ROOM, -5.0, -4.0, 0.0, 5.0, 4.0, 3.0)
    for cx, cy in ((2.5, 1.8), (-2.2, -1.9)):
        s.add(OBB, cx + rng.uniform(-0.4, 0.4), cy + rng.uniform(-0.4, 0.4), 0.6,
              rng.uniform(0.4, 0.7), rng.uniform(0.3, 0.6), 0.6, rng.uniform(-0.6, 0.6))
    return s


def tunnel_network(seed: int, length: float = 230.0):
    """Corridor network: floor plane, wall slabs, arched ceilings, rubble boxes and pillars.

    Returns (scene, centreline) where the centreline is a list of (x, y, heading)
    vertices every segment.
    """
    rng = np.random.default_rng(seed)
    s = Scene(name="tunnel")
    s.add(PLANE, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    x, y, h = 0.0, 0.0, 0.0
    verts = [(x, y, h)]
    travelled = 0.0
    first = True
    while travelled < length:
        L = float(rng.uniform(18.0, 32.0))
        width = float(rng.uniform(3.0, 5.0))
        wall_h = float(rng.uniform(2.2, 3.0))
        ch, sh = math.cos(h), math.sin(h)
        cx, cy = x + 0.5 * L * ch, y + 0.5 * L * sh
        for side in (-1.0, 1.0):
            off = side * (0.5 * width + 0.2)
            wx, wy = cx - off * sh, cy + off * ch
            s.add(OBB, wx, wy, 0.5 * wall_h, 0.5 * L + 0.3, 0.2, 0.5 * wall_h, h)
        # half-tube ceiling resting on the walls
        s.add(ARCH, x, y, wall_h, h, 0.5 * width + 0.01, L)
        if first:
            # dead end behind the start so the first scans see a closed tunnel
            s.add(OBB, x - 0.5 * ch, y - 0.5 * sh, 2.0, 0.2, 0.5 * width + 0.5, 2.0, h)
            first = False
        # rubble boxes along the walls and a few free-standing pillars
        a = 1.5
        while a < L - 1.0:
            side = rng.choice([-1.0, 1.0])
            lat = side * (0.5 * width - rng.uniform(0.25, 0.7))
            bx, by = x + a * ch - lat * sh, y + a * sh + lat * ch
            hx, hy, hz = rng.uniform(0.15, 0.45), rng.uniform(0.15, 0.4), rng.uniform(0.1, 0.5)
            s.add(OBB, bx, by, hz, hx, hy, hz, h + rng.uniform(-0.8, 0.8))
            a += float(rng.uniform(2.0, 4.5))
        x, y = x + L * ch, y + L * sh
        travelled += L
        h = h + float(rng.uniform(-0.5, 0.5))
        verts.append((x, y, h))
    return s, verts


def campus(seed: int, extent: float = 260.0) -> Scene:
    """Outdoor campus: rough ground (5 cm), building facades, poles and trees."""
    rng = np.random.default_rng(seed)
    s = Scene(name="campus")
    s.add(HFIELD, 0.05, 0.5, float(seed % 1000003), 0.0)
    # buildings on both sides of a loop of streets around the origin
    for k in range(60):
        ang = rng.uniform(0, 2 * math.pi)
        rad = rng.uniform(20.0, extent)
        bx, by = rad * math.cos(ang), rad * math.sin(ang)
        if abs(by) < 12.0 or abs(bx) < 12.0:
            continue  # keep the streets along the axes clear
        s.add(OBB, bx, by, 8.0, rng.uniform(4, 15), rng.uniform(4, 15), 8.0, rng.uniform(-0.3, 0.3))
    for k in range(160):
        px = rng.uniform(-extent, extent)
        py = rng.choice([-1.0, 1.0]) * rng.uniform(5.0, 11.0)
        if rng.random() < 0.5:
            px, py = py, px
        s.add(VCYL, px, py, rng.uniform(0.1, 0.5), -1.0, rng.uniform(3.0, 9.0))
    return s


def forest(seed: int, extent: float = 60.0, min_dist: float = 3.0) -> Scene:
    """Poisson-disc trunks (r 0.1-0.4 m) on uneven height-field terrain."""
    rng = np.random.default_rng(seed)
    s = Scene(name="forest")
    s.add(HFIELD, 0.6, 5.0, float(seed % 1000003), 0.0)
    pts = []
    tries = 0
    while tries < 30000 and len(pts) < 900:
        tries += 1
        p = rng.uniform(-extent, extent, size=2)
        if np.hypot(*p) < 2.5:
            continue  # keep the sensor's start free
        if pts and np.min(np.hypot(*(np.asarray(pts) - p).T)) < min_dist:
            continue
        pts.append(p)
    for p in pts:
        gz = s.ground_height(float(p[0]), float(p[1]))
        s.add(VCYL, float(p[0]), float(p[1]), rng.uniform(0.1, 0.4), gz - 1.0, gz + rng.uniform(6.0, 18.0))
    return s


def road(seed: int, length: float = 400.0) -> Scene:
    """Straight road with buildings, parked cars and poles."""
    rng = np.random.default_rng(seed)
    s = Scene(name="road")
    s.add(PLANE, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    x = -50.0
    while x < length:
        for side in (-1.0, 1.0):
            w = rng.uniform(8, 25)
            s.add(OBB, x + w / 2, side * rng.uniform(14, 22), 6.0, w / 2, rng.uniform(3, 6), 6.0, 0.0)
            if rng.random() < 0.6:
                s.add(OBB, x + rng.uniform(0, w), side * rng.uniform(4.0, 5.5), 0.75, 2.2, 0.9, 0.75,
                      rng.uniform(-0.1, 0.1))
            if rng.random() < 0.7:
                s.add(VCYL, x + rng.uniform(0, w), side * rng.uniform(7.0, 9.0), 0.15, -1.0, 6.0)
        x += w + rng.uniform(1, 6)
    return s


# ----------------------------------------------------------------------------- scans

def scan(scene: Scene, lidar: Lidar, P_w_s: np.ndarray, rng: np.random.Generator | None,
         return_truth: bool = False):
    """Ray-cast one sweep; Gaussian range noise and Bernoulli dropouts from ``rng``."""
    d_s = lidar.directions()
    R, t = P_w_s[:, :3], P_w_s[:, 3]
    rng_t, nrm_w, ids = scene.cast(t, d_s @ R.T, lidar.r_max * 1.2)
    n = d_s.shape[0]
    valid = (rng_t >= lidar.r_min) & (rng_t <= lidar.r_max)
    rr = rng_t.copy()
    if rng is not None:
        if lidar.sigma > 0:
            rr = rr + lidar.sigma * rng.standard_normal(n)
        if lidar.dropout > 0:
            valid &= rng.random(n) >= lidar.dropout
    valid &= (rr >= lidar.r_min) & (rr <= lidar.r_max)
    out = np.zeros((n, 4), dtype=np.float32)
    xyz = (d_s * rr[:, None]).astype(np.float32)
    out[valid, :3] = xyz[valid]
    out[valid, 3] = 1.0
    if return_truth:
        return out, (nrm_w @ R).astype(np.float64), ids
    return out


def render_keyframe(scene: Scene, kf: Pano, P_w_kf: np.ndarray):
    """Exact depth (range) and sensor-frame normals at every keyframe pixel centre.

    Returns (depth (rows, cols) FP64, normals (rows, cols, 3) FP64, hit ids).
    Pixels without a return in [r_min, r_max] get depth 0.
    """
    d_s = kf.pixel_dirs().reshape(-1, 3)
    R, t = P_w_kf[:, :3], P_w_kf[:, 3]
    rng_t, nrm_w, ids = scene.cast(t, d_s @ R.T, float(kf.r_max) * 1.2)
    ok = (rng_t >= float(kf.r_min)) & (rng_t <= float(kf.r_max))
    depth = np.where(ok, rng_t, 0.0)
    nrm = np.where(ok[:, None], nrm_w @ R, 0.0)
    return depth.reshape(kf.rows, kf.cols), nrm.reshape(kf.rows, kf.cols, 3), ids.reshape(kf.rows, kf.cols)


# ----------------------------------------------------------------------------- trajectories

def _smooth_noise(rng: np.random.Generator, n: int, amp: float, periods=(40.0, 97.0, 211.0)):
    s = np.arange(n, dtype=np.float64)
    out = np.zeros(n)
    for p in periods:
        out += np.sin(2 * math.pi * s / p + rng.uniform(0, 2 * math.pi))
    return amp * out / len(periods)


def tunnel_trajectory(verts, n_scans: int, step: float, rng: np.random.Generator,
                      height: float = 1.0) -> list:
    """Poses along the corridor centreline at ``step`` metres per scan, with smooth jitter."""
    pts = np.array([(v[0], v[1]) for v in verts])
    seg = np.diff(pts, axis=0)
    seglen = np.hypot(seg[:, 0], seg[:, 1])
    cum = np.concatenate([[0.0], np.cumsum(seglen)])
    heads = np.arctan2(seg[:, 1], seg[:, 0])
    yaw_j = _smooth_noise(rng, n_scans, math.radians(2.0))
    pitch_j = _smooth_noise(rng, n_scans, math.radians(1.0))
    lat_j = _smooth_noise(rng, n_scans, 0.25)
    poses = []
    for k in range(n_scans):
        sdist = 2.0 + k * step
        i = int(np.searchsorted(cum, sdist, side="right") - 1)
        i = min(max(i, 0), len(seglen) - 1)
        f = sdist - cum[i]
        hd = heads[i]
        # blend headings over 2 m around each vertex
        if i + 1 < len(heads) and seglen[i] - f < 1.0:
            w = (1.0 - (seglen[i] - f)) / 2.0
            hd = hd + w * math.remainder(heads[i + 1] - hd, 2 * math.pi)
        if i > 0 and f < 1.0:
            w = (1.0 - f) / 2.0
            hd = hd + w * math.remainder(heads[i - 1] - hd, 2 * math.pi)
        c, s_ = math.cos(heads[i]), math.sin(heads[i])
        x = pts[i, 0] + f * c - lat_j[k] * s_
        y = pts[i, 1] + f * s_ + lat_j[k] * c
        R = rot_zyx(hd + yaw_j[k], pitch_j[k], 0.3 * pitch_j[k])
        poses.append(pose(R, [x, y, height]))
    return poses


def line_trajectory(n_scans: int, step: float, rng: np.random.Generator, y0: float = 0.0,
                    height: float = 1.8, scene: Scene | None = None, heading: float = 0.0) -> list:
    yaw_j = _smooth_noise(rng, n_scans, math.radians(2.0))
    pitch_j = _smooth_noise(rng, n_scans, math.radians(0.7))
    poses = []
    for k in range(n_scans):
        d = k * step
        x, y = d * math.cos(heading) - y0 * math.sin(heading), d * math.sin(heading) + y0 * math.cos(heading)
        z = height + (scene.ground_height(x, y) if scene is not None else 0.0)
        poses.append(pose(rot_zyx(heading + yaw_j[k], pitch_j[k], 0.5 * pitch_j[k]), [x, y, z]))
    return poses
