"""The five workloads the method is exercised on, by what they are and their sizes.

room_200k      200k points, one 8x6x3 m room, 2 scanners; one 256x256 view, cell 0.5 m,
               n_levels 3, filter_strength 1.0; 3-level U-Net 16/32/64 in FP32.
multiroom_20M  20M points, 12x12x4 m, 3x3 rooms, 8 scanners; 16 poses at 1920x1080,
               cell 0.25 m, n_levels 5, filter_strength in {0.5, 1.0}; 4-level U-Net
               32/64/128/256 (FP32 plain path, BF16 and FP8 variants).
multiroom_100M 100M points, 30x30x6 m, 5x5 rooms, 24 scanners; 8 views per launch at
               1920x1080, BF16 U-Net, cell 0.25 m.
serve_100M     the 100M scene resident; 2000 Poisson requests at mixed resolutions
               (1280x720, 1920x1080, 2560x1440), n_levels 4..6, filter_strength U[0.5,1.5].
"""
from __future__ import annotations

import dataclasses

SEED_SCENE, SEED_WEIGHTS, SEED_POSES, SEED_REQUESTS = 0, 1, 2, 3


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_points: int
    scene: str              # "room" or "multiroom"
    scene_kw: dict
    W: int
    H: int
    cell: float
    n_levels: int
    fs: tuple
    unet_ch: tuple
    n_views: int


ROOM_200K = Workload("room_200k", 200_000, "room", {}, 256, 256, 0.5, 3, (1.0,),
                     (16, 32, 64), 1)
MULTIROOM_20M = Workload("multiroom_20M", 20_000_000, "multiroom",
                         dict(extent=(12.0, 12.0, 4.0), rooms=(3, 3), n_boxes=30, n_scanners=8),
                         1920, 1080, 0.25, 5, (0.5, 1.0), (32, 64, 128, 256), 16)
MULTIROOM_100M = Workload("multiroom_100M", 100_000_000, "multiroom",
                          dict(extent=(30.0, 30.0, 6.0), rooms=(5, 5), n_boxes=75, n_scanners=24),
                          1920, 1080, 0.25, 5, (1.0,), (32, 64, 128, 256), 8)


def make_scene(w: Workload, n_points=None, device="cpu"):
    from .scene import room_scene, multiroom_scene
    n = w.n_points if n_points is None else n_points
    if w.scene == "room":
        return room_scene(n_points=n, seed=SEED_SCENE, device=device, **w.scene_kw)
    return multiroom_scene(n_points=n, seed=SEED_SCENE, device=device, **w.scene_kw)
