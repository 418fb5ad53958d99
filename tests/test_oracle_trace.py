"""Pins for the oracle's ray casting, G-buffer, soft shadows and AO.

Section 3.1 (soft shadow, Fig. 1), Section 3.2 (AO, Eqs. 1-3).  Every
expected value below is a closed form, an independent library routine
(numpy.linalg.solve) or an exact special case; Monte Carlo checks use
binomial 4.5-sigma bounds.
"""
import math

import numpy as np
import pytest

import workloads as wl

BIG = 1.0e4


def _quad(corners, mesh_id):
    return wl.scene_quad(corners, mesh_id)


def _floor(mesh_id=0, half=BIG):
    return _quad([[-half, 0, -half], [-half, 0, half], [half, 0, half], [half, 0, -half]], mesh_id)


def _down_camera(x, y, z, size=256):
    return wl.look_at((x, y, z), (x, 0.0, z), size, size)


def test_mt_matches_linear_solve(orc):
    """Closest hit of the brute-force caster equals the smallest positive
    t of o + t d = v0 + u e1 + v e2 solved by numpy.linalg.solve."""
    r = np.random.default_rng(7)
    for trial in range(30):
        nt = 12
        verts = r.uniform(-2, 2, (nt * 3, 3)).astype(np.float32)
        scene = dict(vertices=verts, indices=np.arange(nt * 3, dtype=np.uint32).reshape(nt, 3),
                     mesh_ids=np.arange(nt, dtype=np.uint32))
        S = orc.Scene(scene)
        tri = verts.astype(np.float64).reshape(nt, 3, 3)
        for _ in range(20):
            o = r.uniform(-3, 3, 3)
            d = r.normal(size=3)
            best_t, best_i = math.inf, -1
            for i in range(nt):
                A = np.stack([-d, tri[i, 1] - tri[i, 0], tri[i, 2] - tri[i, 0]], 1)
                t, u, v = np.linalg.solve(A, o - tri[i, 0])
                if t > 0 and u >= 0 and v >= 0 and u + v <= 1 and t < best_t:
                    best_t, best_i = t, i
            res = orc.cast(S, o, d)
            if best_i < 0:
                assert not res["hit"]
            else:
                assert res["hit"] and res["tri"] == best_i
                assert abs(res["t"] - best_t) <= 1e-9 * max(1.0, best_t)


def test_gbuffer_plane_depth_normal(orc):
    """Camera straight above a plane: linear depth = height, normal = +y,
    mesh id of the plane; a pixel outside the plane is background."""
    S = orc.Scene(_floor(mesh_id=5, half=3.0))
    cam = _down_camera(0.3, 2.5, -0.2, 64)
    tr = orc.trace(S, cam, orc.TraceParams())
    fg = tr["mesh"] != 0xFFFFFFFF
    assert fg.all()
    assert np.allclose(tr["depth"], 2.5, rtol=1e-6)
    assert np.allclose(tr["normal"], [0, 1, 0], atol=1e-12)
    assert (tr["mesh"] == 5).all()
    # a camera looking away from every triangle sees background only
    cam2 = wl.look_at((0, 1, 0), (0, 2, 0.01), 16, 16)
    tr2 = orc.trace(S, cam2, orc.TraceParams())
    assert (tr2["mesh"] == 0xFFFFFFFF).all() and np.isinf(tr2["depth"]).all()
    assert (tr2["ao_count"] == 1).all() and (tr2["shadow_mask"] == 1).all()


def test_gbuffer_normal_faces_camera(orc):
    """The stored normal is the geometric normal flipped toward the viewer
    (a floor seen from below)."""
    S = orc.Scene(_floor(half=3.0))
    cam = wl.look_at((0, -2, 0), (0, 0, 0), 16, 16)
    tr = orc.trace(S, cam, orc.TraceParams())
    assert np.allclose(tr["normal"], [0, -1, 0], atol=1e-12)


def test_ao_open_plane_is_one(orc):
    """Eq. 3: nothing within r above an open plane => O = N/N = 1."""
    S = orc.Scene(_floor())
    cam = _down_camera(0, 3, 0, 64)
    tr = orc.trace(S, cam, orc.TraceParams(ao_spp=8, ao_radius=5.0))
    assert (tr["ao_count"] == 8).all()
    assert (tr["shadow_mask"] == 1).all()


def test_ao_enclosed_sphere_is_zero(orc):
    """A point inside a closed sphere of diameter < r: every AO ray is
    occluded (O = 0), and so is every shadow ray."""
    S = orc.Scene(wl.scene_enclosing_sphere(radius=0.4, level=3))
    cam = wl.look_at((0.01, 0.02, 0.0), (0.01, 0.02, -1.0), 64, 64)
    tr = orc.trace(S, cam, orc.TraceParams(ao_spp=8, ao_radius=1.0))
    assert (tr["mesh"] == 0).all()
    assert (tr["ao_count"] == 0).all()
    assert (tr["shadow_mask"] == 0).all()


def _binomial_ok(hits, n, p, k=4.5):
    return abs(hits - n * p) <= k * math.sqrt(n * p * (1 - p))


def test_ao_foot_of_infinite_wall_is_half(orc):
    """Floor point next to an (effectively) infinite wall with unbounded AO
    radius: the wall blocks exactly the half-space of directions toward it,
    which carries half the cosine-weighted measure => O = 0.5."""
    wall = _quad([[0, 0, -BIG], [0, BIG, -BIG], [0, BIG, BIG], [0, 0, BIG]], 1)
    S = orc.Scene(wl.merge(_floor(), wall))
    cam = _down_camera(0.6, 1.0, 0.0, 128)
    tp = orc.TraceParams(ao_spp=8, ao_radius=1.0e6)
    tr = orc.trace(S, cam, tp)
    floor = (tr["mesh"] == 0) & (tr["pos"][:, 0] > 1e-3)
    n = int(floor.sum()) * 8
    hits = int(tr["ao_count"][floor].astype(np.int64).sum())
    assert n > 100000
    assert _binomial_ok(hits, n, 0.5)


@pytest.mark.parametrize("h,r", [(0.5, 1.0), (0.5, 0.6), (0.3, 2.0)])
def test_ao_under_ceiling_closed_form(orc, h, r):
    """Floor under a ceiling at height h, AO radius r > h: a ray is
    unoccluded iff h / cos(theta) >= r; under the cosine-weighted pdf
    P(cos(theta) <= c) = c^2, so O = (h / r)^2."""
    ceil = _quad([[-BIG, h, -BIG], [BIG, h, -BIG], [BIG, h, BIG], [-BIG, h, BIG]], 1)
    # a small floor: secondary rays start 16 ulps of the largest vertex
    # coordinate above it, which must stay negligible against h
    S = orc.Scene(wl.merge(_floor(half=4.0), ceil))
    cam = _down_camera(0.0, h / 2, 0.0, 128)
    tr = orc.trace(S, cam, orc.TraceParams(ao_spp=8, ao_radius=r))
    fl = tr["mesh"] == 0
    n = int(fl.sum()) * 8
    hits = int(tr["ao_count"][fl].astype(np.int64).sum())
    assert _binomial_ok(hits, n, (h / r) ** 2)


def test_ao_radius_shorter_than_ceiling_is_one(orc):
    """A hit beyond the radius is ignored (Section 3.2)."""
    ceil = _quad([[-BIG, 0.5, -BIG], [BIG, 0.5, -BIG], [BIG, 0.5, BIG], [-BIG, 0.5, BIG]], 1)
    S = orc.Scene(wl.merge(_floor(half=4.0), ceil))
    cam = _down_camera(0.0, 0.25, 0.0, 64)
    tr = orc.trace(S, cam, orc.TraceParams(ao_spp=8, ao_radius=0.49))
    assert (tr["ao_count"][tr["mesh"] == 0] == 8).all()


def _disk_fraction_below(a):
    """Fraction of the unit disk with x < a (circular segment)."""
    a = np.clip(a, -1.0, 1.0)
    return 1.0 - (np.arccos(a) - a * np.sqrt(1 - a * a)) / math.pi


def test_soft_shadow_penumbra_closed_form(orc):
    """Section 3.1 / Fig. 1b: a half-plane occluder at height H with its edge
    along z through x = 0 and a light straight above with cone half angle
    theta.  The jittered ray from floor point x0 crosses the occluder plane at
    x0 + H tan(theta) x_s (tangent-disk form), so the lit probability is one
    minus the circular-segment fraction of the disk with x_s < -x0 / (H tan)."""
    Hh, deg = 1.0, 5.0
    occ = _quad([[-BIG, Hh, -BIG], [0, Hh, -BIG], [0, Hh, BIG], [-BIG, Hh, BIG]], 1)
    S = orc.Scene(wl.merge(_floor(half=4.0), occ))
    cam = _down_camera(0.0, 0.5, 0.0, 128)
    T, _ = orc.onb_f32(np.array([0, 1, 0], np.float32))
    assert abs(abs(float(T[0])) - 1) < 1e-7
    tan_t = math.tan(math.radians(deg))
    lit, expect, var = 0, 0.0, 0.0
    counts = np.zeros(10)
    exp_b = np.zeros(10)
    var_b = np.zeros(10)
    for frame in range(6):
        tp = orc.TraceParams(light_dirs=[(0, 1, 0)], cone_half_angle_deg=[deg], frame=frame)
        tr = orc.trace(S, cam, tp)
        fl = tr["mesh"] == 0
        x0 = tr["pos"][fl, 0]
        a = -x0 / (Hh * tan_t * float(T[0]))
        p = 1.0 - _disk_fraction_below(a)
        b = (tr["shadow_mask"][fl] & 1).astype(float)
        lit += b.sum()
        expect += p.sum()
        var += (p * (1 - p)).sum()
        inside = np.abs(a) < 1
        idx = np.clip(((a[inside] + 1) * 5).astype(int), 0, 9)
        np.add.at(counts, idx, b[inside])
        np.add.at(exp_b, idx, p[inside])
        np.add.at(var_b, idx, (p * (1 - p))[inside])
    assert abs(lit - expect) <= 4.5 * math.sqrt(var)
    assert np.all(np.abs(counts - exp_b) <= 4.5 * np.sqrt(var_b) + 1)
    # the umbra side (a >= 1) is always dark, the lit side (a <= -1) always lit


def test_hard_shadow_when_cone_is_zero(orc):
    """Cone angle 0 => every shadow ray points at the light centre (hard
    shadow, Fig. 1a): the mask equals one unjittered ray per pixel."""
    s = wl.scene_boxes()
    S = orc.Scene(s)
    cam = wl.boxes_camera(48, 48)
    l = np.array([0.3, 1.0, 0.2]) / np.linalg.norm([0.3, 1.0, 0.2])
    tr0 = orc.trace(S, cam, orc.TraceParams(cone_half_angle_deg=[0.0], frame=0))
    tr1 = orc.trace(S, cam, orc.TraceParams(cone_half_angle_deg=[0.0], frame=1, seed=99))
    assert (tr0["shadow_mask"] == tr1["shadow_mask"]).all()
    fg = np.nonzero(tr0["mesh"] != 0xFFFFFFFF)[0][::7]
    lf = l.astype(np.float32).astype(np.float64)
    for i in fg:
        X = tr0["pos"][i]
        res = orc.cast(S, X, lf, tmin=1e-9 * (1 + np.abs(X).max()), any_hit=True)
        assert (tr0["shadow_mask"][i] & 1) == (0 if res["hit"] else 1)


def test_ao_count_range_eq3(orc):
    """Eq. 3: 0 <= N_unoccluded <= N, so O lies in [0, 1]."""
    S = orc.Scene(wl.scene_boxes())
    tr = orc.trace(S, wl.boxes_camera(64, 64), orc.TraceParams(ao_spp=13))
    assert tr["ao_count"].max() <= 13
    assert tr["ao_count"].min() < 13        # some occlusion near the boxes


def test_ambiguity_margin(orc):
    """The grazing classification: a ray through a triangle's centroid is
    unambiguous, one through an edge midpoint or a hair outside it is
    ambiguous, one far outside is not."""
    S = orc.Scene(_quad([[0, 0, 0], [1, 0, 0], [1, 0, 1], [0, 0, 1]], 0))
    d = np.array([0.0, -1.0, 0.0])
    cases = [((0.6, 1, 0.3), False), ((0.5, 1, 0.5), True),    # diagonal edge of both triangles
             ((1.0, 1, 0.5), True), ((1.0 + 1e-6, 1, 0.5), True), ((1.0 + 1e-4, 1, 0.5), False), ((1.2, 1, 0.5), False)]
    for o, amb in cases:
        for any_hit in (False, True):
            assert orc.cast(S, np.array(o, float), d, any_hit=any_hit)["ambiguous"] == amb, (o, any_hit)
