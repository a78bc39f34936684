"""Seeded synthetic LiDAR range-image pairs.

This package is the only code shared by the CPU oracle and the CUDA path: it
produces *inputs* (sensor lookup tables, range images, ground-truth poses) and
holds none of the registration method's arithmetic.  It simulates a spinning
LiDAR by analytic ray casting against procedural scenes (ground plane, boxes,
cylinders, closed rooms) so that the paper's missing datasets (its own Ouster
OS0-128 sequences and KITTI) can be stood in for with seeded data of the same
shape, range mix and invalid-pixel ratio.
"""
from .luts import uniform_phi, hdl64_like_phi, zero_theta, random_theta
from .scenes import Sensor, Scene, outdoor_scene, indoor_scene, raycast, random_delta_pose
from .configs import CONFIGS, PairConfig, make_pair, make_pairs, MIXED_KINDS, mixed_batch_plan

__all__ = [
    "uniform_phi", "hdl64_like_phi", "zero_theta", "random_theta",
    "Sensor", "Scene", "outdoor_scene", "indoor_scene", "raycast", "random_delta_pose",
    "CONFIGS", "PairConfig", "make_pair", "make_pairs", "MIXED_KINDS", "mixed_batch_plan",
]
