"""Seeded render-request streams for the serving workload.

Requests arrive as a Poisson process of rate `lam` (exponential inter-arrival times),
each with its own camera pose, a resolution drawn uniformly from a set, a pyramid depth
n_levels drawn uniformly from a range and filter_strength uniform in [fs_lo, fs_hi].
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .camera import View, random_poses

RESOLUTIONS = ((1280, 720), (1920, 1080), (2560, 1440))


@dataclasses.dataclass(frozen=True)
class Request:
    arrival_s: float
    view: View
    W: int
    H: int
    n_levels: int
    fs: float


def request_stream(scene, n, lam=None, seed=3, resolutions=RESOLUTIONS, levels=(4, 6),
                   fs_range=(0.5, 1.5)):
    """n requests; lam=None puts every arrival at t=0 (closed-loop)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if lam is None:
        arrivals = np.zeros(n)
    else:
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=n))
    res = rng.integers(0, len(resolutions), size=n)
    nl = rng.integers(levels[0], levels[1] + 1, size=n)
    fs = rng.uniform(*fs_range, size=n).astype(np.float32)
    views = random_poses(scene, n, seed=seed + 1000)
    return [Request(float(arrivals[i]), views[i], resolutions[res[i]][0], resolutions[res[i]][1],
                    int(nl[i]), float(fs[i])) for i in range(n)]
