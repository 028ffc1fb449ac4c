"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This package holds input generation only: the 7-DoF arm description, obstacle
scenes, their occupancy grids and dense distance fields, start configurations
and target-pose paths.  It contains none of the SMPC iteration's arithmetic
(no sampling, rollout, forward kinematics, cost or weighting).  Every value it
hands out is exactly representable in float32, so the FP32 device path and the
FP64 oracle consume bit-identical inputs.

Scene files under ``workloads/scenes/`` (obstacles, start and target
configurations, target poses) are written by ``oracle/make_scenes.py``, which
uses the oracle's forward kinematics for the collision-free and reachability
rejection tests; this package only reads them.
"""
from .robot import panda_robot, default_cost_params, self_collision_pairs, READY_POSE
from .scenes import (
    GridDesc,
    occupancy_grid,
    distance_grid,
    load_scene,
    build_scene_grid,
    scene_names,
    moving_target,
)

__all__ = [
    "panda_robot",
    "default_cost_params",
    "self_collision_pairs",
    "READY_POSE",
    "GridDesc",
    "occupancy_grid",
    "distance_grid",
    "load_scene",
    "build_scene_grid",
    "scene_names",
    "moving_target",
]
