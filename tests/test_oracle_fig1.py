"""The worked example of Section 3.1 / Fig. 1 (tests/golden/fig1_bitmask.json):
one pixel, three lights.  With rays to the light centres light 0 is occluded
and lights 1 and 2 are not (bitmask 0b110); with cone-jittered rays light 0
stays occluded (its occluder spans the cone), light 1 stays free, and light 2
is occluded for some directions only (its occluder covers part of the cone,
not the axis).  The scene below is built to that description."""
import json
import math
import os

import numpy as np

import oracle as orc
import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))


def _quad(center, u, v, mesh):
    c, u, v = (np.asarray(a, np.float64) for a in (center, u, v))
    return wl.scene_quad([c - u - v, c + u - v, c + u + v, c - u + v], mesh)


def _scene():
    s2 = math.sqrt(0.5)
    L0, L2 = np.array([-s2, s2, 0.0]), np.array([s2, s2, 0.0])
    t0, t2 = np.array([s2, s2, 0.0]), np.array([-s2, s2, 0.0])   # in-plane perpendiculars
    z = np.array([0.0, 0.0, 1.0])
    ground = wl.scene_quad([[-0.5, 0, -0.5], [0.5, 0, -0.5], [0.5, 0, 0.5], [-0.5, 0, 0.5]], 0)
    # light 0: a square 2 units out along L0, 2 x 2 across its cone (radius 0.35 there)
    occ0 = _quad(2.0 * L0, 1.0 * t0, 1.0 * z, 1)
    # light 2: a square 2 units out along L2 covering z in [0.05, 1.05] only
    occ2 = _quad(2.0 * L2 + 0.55 * z, 1.0 * t2, 0.5 * z, 2)
    return wl.merge(ground, occ0, occ2), [tuple(L0), (0.0, 1.0, 0.0), tuple(L2)]


def test_fig1_bitmask_hard_and_soft():
    gold = json.load(open(os.path.join(HERE, "golden", "fig1_bitmask.json")))
    s, lights = _scene()
    sc = orc.Scene(s)
    cam = wl.look_at((0.2, 5.0, 0.001), (0.2, 0.0, 0.0), 9, 9)   # off the ground quad's diagonal
    pix = np.array([[4, 4]])
    hard = orc.trace(sc, cam, orc.TraceParams(light_dirs=lights, cone_half_angle_deg=[0.0] * 3), pixels=pix)
    assert hard["mesh"][0] == 0 and hard["amb_shadow"][0] == 0
    assert int(hard["shadow_mask"][0]) == gold["hard"]["bitmask"]
    bits = []
    for f in range(64):
        tr = orc.trace(sc, cam, orc.TraceParams(light_dirs=lights, cone_half_angle_deg=[10.0] * 3, frame=f),
                       pixels=pix)
        assert tr["amb_shadow"][0] == 0
        bits.append([(int(tr["shadow_mask"][0]) >> k) & 1 for k in range(3)])
    bits = np.array(bits)
    assert (bits[:, 0] == 0).all()          # light 0: occluded for every direction
    assert (bits[:, 1] == 1).all()          # light 1: free for every direction
    f2 = bits[:, 2].mean()                  # light 2: penumbra
    assert 0.3 < f2 < 0.9, f2
