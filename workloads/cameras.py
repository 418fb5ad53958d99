"""Seeded cameras and camera paths.

A camera is a pinhole with an orthonormal basis (forward, right, up), a
vertical field of view and an image size; the basis is built here once
(look-at) and handed as float32 values to both the CUDA path and the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .scenes import rng_for


@dataclass
class Camera:
    pos: np.ndarray        # float32[3]
    forward: np.ndarray    # float32[3], unit
    right: np.ndarray      # float32[3], unit
    up: np.ndarray         # float32[3], unit
    tan_half_fov_y: float  # float32 value
    width: int
    height: int

    def as_floats(self) -> np.ndarray:
        """13 float32 values: pos, forward, right, up, tan(fov_y / 2)."""
        return np.concatenate([self.pos, self.forward, self.right, self.up,
                               [self.tan_half_fov_y]]).astype(np.float32)


def look_at(pos, target, width, height, fov_y_deg=60.0, world_up=(0.0, 1.0, 0.0)) -> Camera:
    p = np.asarray(pos, np.float64)
    f = np.asarray(target, np.float64) - p
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(world_up, np.float64))
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(f, np.array([0.0, 0.0, 1.0]))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    u /= np.linalg.norm(u)
    t = np.float32(math.tan(math.radians(fov_y_deg) / 2.0))
    return Camera(p.astype(np.float32), f.astype(np.float32), r.astype(np.float32),
                  u.astype(np.float32), float(t), int(width), int(height))


def boxes_camera(width=256, height=256) -> Camera:
    """Camera for the 194-triangle box scene: (0, 6, 12) looking at the origin."""
    return look_at((0.0, 6.0, 12.0), (0.0, 0.0, 0.0), width, height)


def orbit_path(n_frames, width, height, radius=12.0, height_y=6.0, degrees=6.0, start_deg=0.0):
    """Slow orbit around the origin (small per-frame motion for the box scene)."""
    cams = []
    for k in range(n_frames):
        a = math.radians(start_deg + degrees * k / max(1, n_frames - 1))
        cams.append(look_at((radius * math.sin(a), height_y, radius * math.cos(a)),
                            (0.0, 0.0, 0.0), width, height))
    return cams


def _catmull_rom(p0, p1, p2, p3, t):
    t2, t3 = t * t, t * t * t
    return 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2
                  + (-p0 + 3 * p1 - 3 * p2 + p3) * t3)


def spline_path(terrain, n_frames=60, width=1920, height=1080, index=1, stream=0,
                spacing=6.0):
    """60-frame seeded Catmull-Rom camera path over 8 control points.

    Control points are ``spacing`` units apart with a heading that turns by
    U[-30, 30] degrees per point, at 5-20 units above the terrain.  The frames
    sweep the five inner segments uniformly in the spline parameter; the camera
    looks ahead along the path and 25 degrees down.
    """
    r = rng_for(index * 1000 + 17 + stream)
    lim = terrain.extent - 40.0
    p = r.uniform(-lim / 2, lim / 2, 2)
    heading = r.uniform(0, 2 * math.pi)
    ctrl = []
    for _ in range(8):
        y = terrain.height_at(p[0], p[1]) + r.uniform(5.0, 20.0)
        ctrl.append(np.array([p[0], y, p[1]]))
        heading += math.radians(r.uniform(-30.0, 30.0))
        p = p + spacing * np.array([math.cos(heading), math.sin(heading)])
    ctrl = np.array(ctrl)

    def at(s):
        seg = min(int(s), 4)
        t = s - seg
        i = seg + 1
        return _catmull_rom(ctrl[i - 1], ctrl[i], ctrl[i + 1], ctrl[i + 2], t)

    cams = []
    for k in range(n_frames):
        s = 5.0 * k / n_frames
        pos = at(s)
        ahead = at(min(s + 0.25, 4.999)) - pos
        ahead[1] = 0.0
        if np.linalg.norm(ahead) < 1e-6:
            ahead = np.array([1.0, 0.0, 0.0])
        ahead /= np.linalg.norm(ahead)
        d = ahead * math.cos(math.radians(25)) - np.array([0, 1.0, 0]) * math.sin(math.radians(25))
        cams.append(look_at(pos, pos + d, width, height))
    return cams
