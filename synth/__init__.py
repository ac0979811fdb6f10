"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the benchmark.

This package generates inputs only: LiDAR-like coloured point clouds, camera poses and
intrinsics, U-Net weights and request streams.  It holds none of the render method's
arithmetic (no projection, culling, filtering or convolution), so the oracle and the
CUDA path can both consume it without sharing any of the method's code.
"""
from .scene import Scene, room_scene, multiroom_scene, GEO_OFFSET
from .camera import Intrinsics, View, intrinsics_for, random_poses
from .weights import unet_layer_shapes, unet_weights
from .requests import Request, request_stream
from . import workloads

__all__ = [
    "Scene", "room_scene", "multiroom_scene", "GEO_OFFSET",
    "Intrinsics", "View", "intrinsics_for", "random_poses",
    "unet_layer_shapes", "unet_weights",
    "Request", "request_stream", "workloads",
]
