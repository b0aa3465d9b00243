"""Seeded synthetic inputs for DARE: phantom, tracked sweeps, reslice poses.

This module generates inputs only.  It holds none of the reconstruction or
reslicing arithmetic; the CUDA library and the CPU oracle both consume what it
produces.  The paper's phantom and human datasets (Sec. 2.2) are not
available, so a seeded phantom with Rayleigh speckle, specular ellipsoid
shells and tubular vessels stands in for them, imaged by linear freehand
sweeps with tracking jitter (the acquisition set-up of Sec. 2.1/2.2: a linear
array tracked by an optical tracker).

Conventions shared by every consumer (they are input semantics, not method):
  * poses are row-major 4x4 float64 rigid transforms, image -> world, in mm;
  * image axes: x = lateral, y = beam/depth, z = elevation = x cross y;
  * pixel (u, v) of a W x H frame sits at image point ((u-(W-1)/2) sx, v sy, 0);
  * a grid is (dims (nx, ny, nz), spacing h, vol_to_world 4x4); voxel i's
    centre is vol_to_world @ (i h).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        from . import _build
        path = _build.build()
        lib = ctypes.CDLL(path)
        d = ctypes.POINTER(ctypes.c_double)
        lib.synth_render.argtypes = [
            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
            d, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
            ctypes.c_int32, d, ctypes.c_int32, ctypes.c_int32, d, ctypes.POINTER(ctypes.c_uint8)]
        lib.synth_render.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------- rotations

def rot_axis_angle(axis, angle_rad):
    axis = np.asarray(axis, dtype=np.float64)
    n = np.linalg.norm(axis)
    if n == 0:
        return np.eye(3)
    k = axis / n
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle_rad) * K + (1 - math.cos(angle_rad)) * (K @ K)


def random_rotation(rng):
    """Uniform random rotation (Shoemake's method from a uniform unit quaternion)."""
    u1, u2, u3 = rng.random(3)
    w = math.sqrt(1 - u1) * math.sin(2 * math.pi * u2)
    x = math.sqrt(1 - u1) * math.cos(2 * math.pi * u2)
    y = math.sqrt(u1) * math.sin(2 * math.pi * u3)
    z = math.sqrt(u1) * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def make_pose(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def probe_rotation(tilt_deg):
    """Image->world rotation of a probe swept along world +y, beam tilted about y.

    At tilt 0: lateral = +x, beam = -z, elevation = +y (the sweep direction).
    """
    base = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [0.0, -1.0, 0.0]])  # columns x_w, -z_w, y_w
    return rot_axis_angle([0, 1, 0], math.radians(tilt_deg)) @ base


# ---------------------------------------------------------------- phantom

@dataclass
class Phantom:
    seed: int
    sigma: float = 40.0          # Rayleigh speckle scale
    cell_mm: float = 0.1         # speckle lattice cell
    sigma_t: float = 0.3         # specular profile width (mm)
    echo_gain: float = 200.0     # specular echo amplitude
    shells: np.ndarray = field(default_factory=lambda: np.zeros((0, 15)))
    vessels: np.ndarray = field(default_factory=lambda: np.zeros((0, 7)))
    n_pts: int = 2


def make_phantom(seed, extent_mm, n_shells, n_vessels, vessel_pts=5):
    """Seeded phantom inside a cube of side extent_mm centred at the world origin."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0xF1A5]))
    half = 0.5 * extent_mm
    smax = min(15.0, extent_mm / 4.0)
    smin = min(3.0, 0.5 * smax)
    shells = np.zeros((n_shells, 15))
    for k in range(n_shells):
        shells[k, 0:3] = rng.uniform(-0.5 * half, 0.5 * half, 3)
        shells[k, 3:6] = rng.uniform(smin, smax, 3)
        shells[k, 6:15] = random_rotation(rng).reshape(-1)
    vessels = np.zeros((n_vessels, 1 + 3 * vessel_pts))
    for k in range(n_vessels):
        vessels[k, 0] = rng.uniform(2.0, 5.0) if extent_mm >= 50 else rng.uniform(1.0, 2.5)
        # a gently curving polyline crossing the cube
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
        p0 = rng.uniform(-0.3 * half, 0.3 * half, 3) - a * 1.2 * half
        wig = rng.normal(size=3)
        wig -= wig.dot(a) * a
        wig /= max(np.linalg.norm(wig), 1e-12)
        for i in range(vessel_pts):
            s = i / (vessel_pts - 1)
            p = p0 + a * 2.4 * half * s + wig * 0.15 * half * math.sin(math.pi * s * 1.5)
            vessels[k, 1 + 3 * i:4 + 3 * i] = p
    speckle_seed = int(rng.integers(0, 2**63 - 1))
    return Phantom(seed=speckle_seed, shells=shells, vessels=vessels, n_pts=vessel_pts)


def render_frames(ph: Phantom, poses, W, H, sx, sy):
    poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(-1, 16))
    n = poses.shape[0]
    out = np.empty((n, H, W), dtype=np.uint8)
    shells = np.ascontiguousarray(ph.shells, dtype=np.float64)
    vessels = np.ascontiguousarray(ph.vessels, dtype=np.float64)
    rc = _lib().synth_render(
        n, W, H, sx, sy, _dp(poses), ph.seed, ph.sigma, ph.cell_mm, ph.sigma_t, ph.echo_gain,
        shells.shape[0], _dp(shells) if shells.size else None,
        vessels.shape[0], ph.n_pts, _dp(vessels) if vessels.size else None,
        out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    if rc != 0:
        raise ValueError(f"synth_render failed ({rc})")
    return out


# ---------------------------------------------------------------- grids, sweeps, poses

@dataclass
class Grid:
    dims: tuple
    spacing: float
    vol_to_world: np.ndarray

    @property
    def extent(self):
        return np.array(self.dims, dtype=np.float64) * self.spacing


def centred_grid(dims, spacing, R=None):
    """Grid whose centre sits at the world origin (optionally rotated by R)."""
    R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
    c = (np.array(dims, dtype=np.float64) - 1) * 0.5 * spacing
    return Grid(tuple(int(d) for d in dims), float(spacing), make_pose(R, -R @ c))


def sweep_poses(seed, sweep_index, n_frames, H, sy, tilt_deg, length_mm,
                jitter_mm=0.1, jitter_deg=0.2, centre=(0.0, 0.0, 0.0)):
    """Linear freehand sweep along world +y through `centre`, beam tilted by tilt_deg.

    The image centre (lateral 0, depth H sy / 2) rides on the track; every
    frame gets Gaussian jitter of jitter_mm per axis and jitter_deg about a
    random axis.
    """
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x5EE9, int(sweep_index)]))
    R0 = probe_rotation(tilt_deg)
    qc = np.array([0.0, 0.5 * H * sy, 0.0])
    ys = np.linspace(-0.5 * length_mm, 0.5 * length_mm, n_frames) if n_frames > 1 else np.zeros(1)
    poses = np.empty((n_frames, 4, 4))
    for k in range(n_frames):
        axis = rng.normal(size=3)
        ang = math.radians(rng.normal() * jitter_deg)
        R = rot_axis_angle(axis, ang) @ R0
        track = np.asarray(centre, dtype=np.float64) + np.array([0.0, ys[k], 0.0])
        t = track - R @ qc + rng.normal(size=3) * jitter_mm
        poses[k] = make_pose(R, t)
    return poses


def plane_pose_centred(R, centre, W, H, sx, sy):
    """Pose whose image centre (lateral 0, depth H sy / 2) lands on `centre`."""
    qc = np.array([0.0, 0.5 * (H - 1) * sy, 0.0])
    return make_pose(R, np.asarray(centre, dtype=np.float64) - R @ qc)


def perturbed_poses(seed, base_poses, n, max_deg, max_mm):
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x9E27]))
    idx = rng.integers(0, len(base_poses), n)
    out = np.empty((n, 4, 4))
    for i, j in enumerate(idx):
        T = base_poses[j]
        Rp = rot_axis_angle(rng.normal(size=3), math.radians(rng.uniform(0, max_deg)))
        d = rng.normal(size=3)
        d *= rng.uniform(0, max_mm) / max(np.linalg.norm(d), 1e-12)
        out[i] = make_pose(Rp @ T[:3, :3], T[:3, 3] + d)
    return out


def random_poses(seed, n, W, H, sx, sy, centre_spread_mm):
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x7A4D]))
    out = np.empty((n, 4, 4))
    for i in range(n):
        R = random_rotation(rng)
        c = rng.uniform(-centre_spread_mm, centre_spread_mm, 3)
        out[i] = plane_pose_centred(R, c, W, H, sx, sy)
    return out


def smooth_trajectory(seed, n, rate_hz, W, H, sx, sy, start_tilts, pos_sigma_mm=20.0,
                      speed_mm_s=50.0, ang_speed_deg_s=30.0, tau_s=0.3):
    """Smooth random walk of probe poses sampled at rate_hz.

    Velocity and angular velocity are Ornstein-Uhlenbeck processes (time
    constant tau_s, stationary scales speed_mm_s and ang_speed_deg_s); the
    position is pulled toward the origin so its spread stays near
    pos_sigma_mm.  The orientation starts at one of the sweep orientations.
    """
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x0B57]))
    dt = 1.0 / rate_hz
    R = probe_rotation(float(rng.choice(np.asarray(start_tilts, dtype=np.float64))))
    x = rng.normal(size=3) * 0.25 * pos_sigma_mm
    v = rng.normal(size=3) * speed_mm_s / math.sqrt(3)
    w = rng.normal(size=3) * math.radians(ang_speed_deg_s) / math.sqrt(3)
    a = math.exp(-dt / tau_s)
    sv = speed_mm_s / math.sqrt(3) * math.sqrt(1 - a * a)
    sw = math.radians(ang_speed_deg_s) / math.sqrt(3) * math.sqrt(1 - a * a)
    spring = (speed_mm_s / max(pos_sigma_mm, 1e-9)) ** 2 * 0.5
    out = np.empty((n, 4, 4))
    for i in range(n):
        out[i] = plane_pose_centred(R, x, W, H, sx, sy)
        v = a * v + sv * rng.normal(size=3) - spring * x * dt
        w = a * w + sw * rng.normal(size=3)
        x = x + v * dt
        R = rot_axis_angle(w, np.linalg.norm(w) * dt) @ R
        # re-orthonormalise against drift
        U, _, Vt = np.linalg.svd(R)
        R = U @ Vt
    return out


# ---------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    grid: Grid
    frame_w: int
    frame_h: int
    frame_px: tuple
    frame_poses: np.ndarray     # (n, 4, 4)
    frames: np.ndarray          # (n, H, W) uint8
    out_w: int
    out_h: int
    out_px: tuple
    reslice_poses: np.ndarray   # (m, 4, 4)
    sweep_tilts: tuple
    phantom: "Phantom" = None   # the scene the frames were rendered from (renders ground truth at any pose)


def tiny_workload(seed=0, render=True):
    """64^3 grid at 0.5 mm; 2 sweeps x 100 frames of 128x128 at 0.25 mm, tilts +-30 deg;
    3 specular shells; 16 reslice poses at 128x128, 0.25 mm (8 within 10 deg /
    3 mm of an acquired frame, 4 within 35 deg / 3 mm, 4 uniformly random)."""
    grid = centred_grid((64, 64, 64), 0.5)
    W = H = 128
    sx = sy = 0.25
    tilts = (30.0, -30.0)
    L = grid.extent[1]
    poses = np.concatenate([sweep_poses(seed, s, 100, H, sy, t, L) for s, t in enumerate(tilts)])
    ph = make_phantom(seed, float(grid.extent[0]), 3, 0)
    frames = render_frames(ph, poses, W, H, sx, sy) if render else None
    rp = np.concatenate([perturbed_poses(seed, poses, 8, 10.0, 3.0),
                         perturbed_poses(seed + 1000, poses, 4, 35.0, 3.0),
                         random_poses(seed, 4, W, H, sx, sy, 6.0)])
    return Workload("dare_64cube_200f_128px", grid, W, H, (sx, sy), poses, frames, W, H, (sx, sy), rp, tilts, ph)


def working_workload(seed=1, n_poses=1000, render=True):
    """256^3 grid at 0.4 mm; 4 sweeps (0, +35, -35, 90 deg) x 400 frames of 256x512
    at 0.2 mm; 8 specular shells and 2 vessels; n_poses reslice poses of 512x512
    at 0.2 mm along a smooth random walk sampled at 1 kHz."""
    grid = centred_grid((256, 256, 256), 0.4)
    W, H = 256, 512
    sx = sy = 0.2
    tilts = (0.0, 35.0, -35.0, 90.0)
    L = grid.extent[1]
    poses = np.concatenate([sweep_poses(seed, s, 400, H, sy, t, L) for s, t in enumerate(tilts)])
    ph = make_phantom(seed, float(grid.extent[0]), 8, 2)
    frames = render_frames(ph, poses, W, H, sx, sy) if render else None
    rp = smooth_trajectory(seed, n_poses, 1000.0, 512, 512, 0.2, 0.2, tilts)
    return Workload("dare_256cube_1600f_512px", grid, W, H, (sx, sy), poses, frames, 512, 512, (0.2, 0.2), rp, tilts,
                    ph)


@dataclass
class BatchVolume:
    grid: Grid
    frame_w: int
    frame_h: int
    frame_px: tuple
    frame_poses: np.ndarray
    frames: np.ndarray
    plane_poses: np.ndarray      # (m, 4, 4)
    plane_sizes: list            # m x (W, H)
    plane_px: tuple


def batched_workload(seed=3, n_volumes=64, frame_step_mm=0.8, px_mm=0.4, plane_px_mm=0.3, render=True):
    """Uneven batch: n_volumes grids with dims drawn uniformly from 96^3 to
    384 x 384 x 256 at 0.4 mm, each scanned by 2-6 linear sweeps (per-volume
    phantom seed, beam tilts in [-40, 40] deg, sometimes 90), each with 8-32
    reslice planes whose sizes are drawn from {128, 256, 512, 640}^2 (square)."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0xBA7C]))
    vols = []
    for k in range(n_volumes):
        dims = (int(rng.integers(96, 385)), int(rng.integers(96, 385)), int(rng.integers(96, 257)))
        grid = centred_grid(dims, 0.4)
        ext = grid.extent
        W = int(math.ceil(ext[0] / px_mm))
        H = int(math.ceil(ext[2] * 1.1 / px_mm))
        n_sweeps = int(rng.integers(2, 7))
        tilts = [float(rng.uniform(-40, 40)) for _ in range(n_sweeps)]
        if rng.random() < 0.3:
            tilts[-1] = 90.0
        n_frames = max(2, int(ext[1] / frame_step_mm))
        vseed = int(rng.integers(0, 2**31 - 1))
        poses = np.concatenate([sweep_poses(vseed, s, n_frames, H, px_mm, t, float(ext[1]), centre=(0.0, 0.0, 0.0))
                                for s, t in enumerate(tilts)])
        ph = make_phantom(vseed, float(min(ext)), 4 + int(rng.integers(0, 5)), 1)
        frames = render_frames(ph, poses, W, H, px_mm, px_mm) if render else None
        m = int(rng.integers(8, 33))
        sizes = [int(rng.choice([128, 256, 512, 640])) for _ in range(m)]
        base = perturbed_poses(vseed, poses, m, 10.0, 3.0)
        planes = np.stack([plane_pose_centred(base[i][:3, :3], base[i][:3, 3] + base[i][:3, :3] @ np.array(
            [0.0, 0.5 * (H - 1) * px_mm, 0.0]), sizes[i], sizes[i], plane_px_mm, plane_px_mm) for i in range(m)])
        vols.append(BatchVolume(grid, W, H, (px_mm, px_mm), poses, frames, planes, [(z, z) for z in sizes],
                                (plane_px_mm, plane_px_mm)))
    return vols
