"""Seeded camera poses and pinhole intrinsics.

Convention (OpenCV): camera x to the right, y down, z forward.  A view is the
world-to-camera rotation R (row-major 3x3, float64) and the camera centre C (float64,
world coordinates), so a world point p has camera coordinates R (p - C).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Intrinsics:
    fx: float
    fy: float
    cx: float
    cy: float
    znear: float = 0.05
    zfar: float = 100.0


@dataclasses.dataclass(frozen=True)
class View:
    R: np.ndarray   # (3, 3) float64, world -> camera rotation
    C: np.ndarray   # (3,) float64, camera centre in world coordinates


def intrinsics_for(W: int, H: int, hfov_deg: float = 60.0, znear=0.05, zfar=100.0) -> Intrinsics:
    """Square pixels, principal point at the image centre, horizontal field of view hfov."""
    f = (W / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return Intrinsics(float(np.float32(f)), float(np.float32(f)), W / 2.0, H / 2.0, znear, zfar)


def look(yaw: float, pitch: float) -> np.ndarray:
    """World-to-camera rotation for a camera looking along (yaw, pitch), world z up."""
    f = np.array([math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch)])
    right = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    down = np.cross(f, right)
    return np.stack([right, down, f])


def random_poses(scene, n: int, seed: int = 2, height=(1.2, 1.8), pitch_deg=15.0):
    """n camera poses in the scene's free space: height U[1.2,1.8] m, yaw U[0,2pi),
    pitch U[-15,15] degrees."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X, Y, _ = scene.extent
    off = np.asarray(scene.offset, dtype=np.float64)
    views = []
    while len(views) < n:
        p = np.array([[rng.uniform(0.3, X - 0.3), rng.uniform(0.3, Y - 0.3), rng.uniform(*height)]])
        yaw = rng.uniform(0.0, 2 * math.pi)
        pitch = math.radians(rng.uniform(-pitch_deg, pitch_deg))
        if not scene.free_space(p, margin=0.3)[0]:
            continue
        C = np.round((p[0] + off) * 4096.0) / 4096.0
        views.append(View(look(yaw, pitch), C))
    return views
