"""Seeded synthetic inputs shared by the CUDA path, the oracle, tests and bench.

Nothing in this package computes any step of the method (no ray casting, no
sampling, no filtering): it only builds triangle soups, cameras and camera
paths from fixed numpy PCG64 seeds.
"""
from .scenes import (SEED_BASE, rng_for, scene_boxes, scene_terrain, scene_quad,  # noqa: F401
                     scene_enclosing_sphere, merge, triangle_soup, box_mesh, icosphere)
from .cameras import Camera, look_at, boxes_camera, orbit_path, spline_path  # noqa: F401
