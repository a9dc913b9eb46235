"""Seeded scene layouts (instances) and camera paths for the workloads.

Workloads (sizes as the crowd / single-asset experiments of Sec. 5 use them, data synthetic):

* ``tiny``: one asset of 100k leaves, one 256x256 camera, horizontal fov 60 deg, distance 3.
* ``orbit``: one asset of 1M leaves, 1920x1080, fov 45 deg (Sec. 5.1), elevation 30 deg,
  8 distances 1.5 * (50/1.5)^(k/7).
* ``crowd``: 10 assets of 1M leaves, 1000 instances on a 200x200 ground, random rotation,
  uniform scale U[0.5, 2]; a 300-frame walk on a circle of radius 60 at eye height 1.7,
  looking along the tangent turned 20 deg inward; 1920x1080, fov 45 deg.

Cameras are OpenCV style (x right, y down, z forward), world z up.  ``world_to_cam`` is the
row-major 3x4 [R | t] that maps world points to camera space.  Intrinsics are float32 values
shared verbatim by both implementations.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    world_to_cam: np.ndarray   # (3, 4) float64
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.01

    @property
    def center(self) -> np.ndarray:
        r = self.world_to_cam[:, :3]
        return -r.T @ self.world_to_cam[:, 3]


@dataclasses.dataclass
class Instances:
    asset: np.ndarray   # (n,) uint32
    rot: np.ndarray     # (n, 3, 3) float64, proper rotations
    trans: np.ndarray   # (n, 3) float64
    scale: np.ndarray   # (n,) float64, uniform scale > 0

    @property
    def n(self) -> int:
        return int(self.asset.shape[0])


def f32(x: float) -> float:
    return float(np.float32(x))


def look_at(eye, target, width, height, fov_x_deg, up=(0.0, 0.0, 1.0), near=0.01) -> Camera:
    """Pinhole camera at ``eye`` looking at ``target``; horizontal field of view in degrees."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    r = np.stack([right, down, fwd])
    w2c = np.concatenate([r, (-r @ eye)[:, None]], axis=1)
    f = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(w2c, f32(f), f32(f), f32(width / 2.0), f32(height / 2.0), width, height, f32(near))


def look_dir(eye, direction, width, height, fov_x_deg, near=0.01) -> Camera:
    return look_at(eye, np.asarray(eye, np.float64) + np.asarray(direction, np.float64),
                   width, height, fov_x_deg, near=near)


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotations from Shoemake quaternions."""
    u = rng.random((n, 3))
    a, b = np.sqrt(1.0 - u[:, 0]), np.sqrt(u[:, 0])
    t1, t2 = 2 * np.pi * u[:, 1], 2 * np.pi * u[:, 2]
    w, x, y, z = b * np.cos(t2), a * np.sin(t1), a * np.cos(t1), b * np.sin(t2)
    r = np.empty((n, 3, 3))
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - w * z)
    r[:, 0, 2] = 2 * (x * z + w * y)
    r[:, 1, 0] = 2 * (x * y + w * z)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - w * x)
    r[:, 2, 0] = 2 * (x * z - w * y)
    r[:, 2, 1] = 2 * (y * z + w * x)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


# ----------------------------------------------------------------------------- tiny / orbit


def single_instance() -> Instances:
    return Instances(np.zeros(1, np.uint32), np.eye(3)[None].copy(), np.zeros((1, 3)), np.ones(1))


def tiny_camera() -> Camera:
    return look_at((0.0, -3.0, 0.0), (0.0, 0.0, 0.0), 256, 256, 60.0)


def orbit_distances() -> list[float]:
    return [1.5 * (50.0 / 1.5) ** (k / 7.0) for k in range(8)]


def orbit_camera(distance: float, width=1920, height=1080, fov_x=45.0, elev_deg=30.0,
                 azim_deg=-90.0) -> Camera:
    e, a = math.radians(elev_deg), math.radians(azim_deg)
    eye = distance * np.array([math.cos(e) * math.cos(a), math.cos(e) * math.sin(a), math.sin(e)])
    return look_at(eye, (0.0, 0.0, 0.0), width, height, fov_x)


# ----------------------------------------------------------------------------- crowd

CROWD_RING = 60.0
CROWD_EYE_H = 1.7
CROWD_FRAMES = 300


def crowd_instances(n: int = 1000, n_assets: int = 10, seed: int = 1000,
                    half_extent: float = 100.0, ring_clear: float = 3.5) -> Instances:
    """Instances on a (2*half_extent)^2 ground; rejected when within ``ring_clear`` of the walk."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xy = np.empty((0, 2))
    while xy.shape[0] < n:
        cand = rng.uniform(-half_extent, half_extent, size=(2 * n, 2))
        keep = np.abs(np.linalg.norm(cand, axis=1) - CROWD_RING) >= ring_clear
        xy = np.concatenate([xy, cand[keep]])
    xy = xy[:n]
    rot = random_rotations(rng, n)
    scale = rng.uniform(0.5, 2.0, size=n)
    asset = rng.integers(0, n_assets, size=n).astype(np.uint32)
    trans = np.concatenate([xy, scale[:, None]], axis=1)   # the unit-sphere asset rests on z = 0
    return Instances(asset, rot, trans, scale)


def crowd_camera(t: int, width=1920, height=1080, fov_x=45.0, frames=CROWD_FRAMES) -> Camera:
    th = 2.0 * math.pi * t / frames
    eye = (CROWD_RING * math.cos(th), CROWD_RING * math.sin(th), CROWD_EYE_H)
    tangent = np.array([-math.sin(th), math.cos(th), 0.0])
    inward = np.array([-math.cos(th), -math.sin(th), 0.0])
    d = math.cos(math.radians(20.0)) * tangent + math.sin(math.radians(20.0)) * inward
    return look_dir(eye, d, width, height, fov_x)


def subset(inst: Instances, idx) -> Instances:
    idx = np.asarray(idx)
    return Instances(inst.asset[idx].copy(), inst.rot[idx].copy(), inst.trans[idx].copy(),
                     inst.scale[idx].copy())
