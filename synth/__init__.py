"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and by the
CPU oracle.

This package draws random numbers and builds scenes, cameras and poses. It holds
none of the rasterizer's arithmetic (no projection, blending or gradients), so it
can feed both sides of a parity comparison without coupling them.
"""

from .scenes import (  # noqa: F401
    Camera,
    Scene,
    tiny_scene,
    fd_scene,
    room_scene,
    two_room_scene,
    room_track_poses,
    circle_poses,
    mixed_resolution_cameras,
    jitter_pose,
    look_at,
    random_targets,
    workload,
)
