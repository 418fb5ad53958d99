"""Pins of the oracle's selective shadow rays (Section 5: a shadow map marks
the pixels whose shadow it cannot decide; only those get rays).

The classification is pinned to things other than itself: the closed-form
shadow map of a plane, planar receivers that can only be lit (or, facing
away, only in umbra), and brute force -- for every pixel the
classification calls lit or umbra, 13 cone rays (the axis and 12 rays on
the cone's rim, where penumbra begins) cast one by one must all agree with
the verdict, and every pixel whose rays disagree must be in the ray mask.
"""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl

LIGHT = (0.3, 1.0, 0.2)


def _onb(L):
    a = np.array([1.0, 0.0, 0.0]) if abs(L[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    T = np.cross(L, a)
    T /= np.linalg.norm(T)
    return T, np.cross(L, T)


def _cone_rays(L, theta, n_rim=12):
    """The cone axis and n_rim directions on the cone's boundary."""
    L = np.asarray(L, np.float64) / np.linalg.norm(L)
    T, B = _onb(L)
    out = [L]
    for k in range(n_rim):
        ph = 2 * math.pi * k / n_rim
        d = L + math.tan(theta) * (math.cos(ph) * T + math.sin(ph) * B)
        out.append(d / np.linalg.norm(d))
    return out


def _tilted_quad():
    return wl.scene_quad([[-5, 0, -5], [5, 0, -5], [5, 4, 5], [-5, 4, 5]], 3)


@pytest.mark.parametrize("light", [LIGHT, (0.0, 1.0, 0.0), (1.0, 0.2, 0.0), (0.0, -1.0, 0.3)])
def test_frame_is_orthonormal_and_covers_the_scene(light):
    s = wl.scene_boxes()
    sc = orc.Scene(s)
    m = orc.ShadowMap(sc, light, 64, full=False)
    f = m.frame_dict()
    L, eu, ev = f["L"], f["eu"], f["ev"]
    assert np.allclose([L @ L, eu @ eu, ev @ ev], 1.0, atol=1e-14)
    assert abs(L @ eu) < 1e-14 and abs(L @ ev) < 1e-14 and abs(eu @ ev) < 1e-14
    assert np.allclose(np.cross(L, eu), ev, atol=1e-14)
    v = s["vertices"].astype(np.float64)
    u, w_ = v @ eu, v @ ev
    span = f["w"] * f["res"]
    assert (u > f["u0"]).all() and (u < f["u0"] + span).all()
    assert (w_ > f["v0"]).all() and (w_ < f["v0"] + span).all()
    assert (f["h"] - v @ L > 0).all()


def test_map_of_a_plane_matches_closed_form():
    """Quad y = 0 over [-10, 10]^2: the texel ray from O along -L meets the
    plane at t = O.y / L.y, inside the quad iff |x|, |z| <= 10."""
    q = wl.scene_quad([[-10, 0, -10], [10, 0, -10], [10, 0, 10], [-10, 0, 10]], 0)
    sc = orc.Scene(q)
    R = 64
    m = orc.ShadowMap(sc, LIGHT, R)
    f = m.frame_dict()
    L = f["L"]
    j, i = np.mgrid[0:R, 0:R]
    O = (f["h"] * L[None, None, :] + (f["u0"] + (i[..., None] + 0.5) * f["w"]) * f["eu"]
         + (f["v0"] + (j[..., None] + 0.5) * f["w"]) * f["ev"])
    t = O[..., 1] / L[1]
    X = O - t[..., None] * L
    inside = (np.abs(X[..., 0]) <= 10) & (np.abs(X[..., 2]) <= 10)
    ok = m.amb == 0
    assert inside.sum() > R * R // 4
    assert np.allclose(m.depth[ok & inside], t[ok & inside], rtol=1e-12)
    assert np.isinf(m.depth[ok & ~inside]).all()


@pytest.mark.parametrize("scene", ["ground", "tilted"])
def test_planar_receivers_are_lit_or_umbra(scene):
    """A lone plane casts no shadow on itself: every pixel it fills is lit
    (no ray); lit from behind, every pixel is in umbra.  A sign error in
    the tangent-plane term, a transposed axis or a missing bias turns
    some of these pixels into rays or into umbra."""
    if scene == "ground":
        s = wl.scene_quad([[-10, 0, -10], [10, 0, -10], [10, 0, 10], [-10, 0, 10]], 0)
        cam = wl.look_at((0.0, 6.0, 9.0), (0.0, 0.0, 0.0), 80, 60)
    else:
        s = _tilted_quad()
        cam = wl.look_at((0.0, 6.0, -8.0), (0.0, 2.0, 0.0), 80, 60)
    sc = orc.Scene(s)
    for light, want in ((LIGHT, orc.CLS_LIT), ((0.3, -1.0, 0.2), orc.CLS_UMBRA)):
        m = orc.ShadowMap(sc, light, 128)
        tp = orc.TraceParams(light_dirs=[light])
        tr = orc.trace_selective(sc, cam, tp, [m])
        fg = np.isfinite(tr["depth"])
        assert fg.sum() > 1000
        c = tr["cls"][fg, 0]
        assert (c == want).all(), np.bincount(c, minlength=3)
        assert (tr["shadow_mask"] == tr["shadow_mask_full"]).all()


def _brute_force_visibility(sc, tr, idx, L, theta):
    """Per pixel: (all 13 cone rays free, all blocked, any ray ambiguous)."""
    rays = _cone_rays(L, theta)
    out = []
    for p in idx:
        X, n = tr["pos"][p], tr["normal"][p]
        o = X + 1e-4 * n
        hits, amb = [], False
        for d in rays:
            if d @ n <= 1e-9:
                hits.append(True)
                continue
            r = orc.cast(sc, o, d, 0.0, math.inf, any_hit=True)
            hits.append(r["hit"])
            amb |= r["ambiguous"]
        out.append((not any(hits), all(hits), amb))
    return out


@pytest.mark.parametrize("deg", [0.5, 3.0])
def test_classification_matches_brute_force_cone(deg):
    """Boxes on a plane (boxes194): lit pixels see the whole cone, umbra
    pixels none of it, and every penumbra pixel is in the ray mask."""
    s = wl.scene_boxes()
    sc = orc.Scene(s)
    cam = wl.boxes_camera(64, 64)
    m = orc.ShadowMap(sc, LIGHT, 512)
    tp = orc.TraceParams(cone_half_angle_deg=[deg])
    tr = orc.trace_selective(sc, cam, tp, [m])
    fg = np.isfinite(tr["depth"]) & (tr["amb_primary"] == 0)
    idx = np.nonzero(fg & (tr["amb_cls"][:, 0] == 0))[0]
    L = np.asarray(LIGHT) / np.linalg.norm(LIGHT)
    vis = _brute_force_visibility(sc, tr, idx, L, math.radians(deg))
    c = tr["cls"][idx, 0]
    n_pen = 0
    for k, (free, blocked, amb) in enumerate(vis):
        if amb:
            continue
        if c[k] == orc.CLS_LIT:
            assert free, (idx[k], c[k])
        elif c[k] == orc.CLS_UMBRA:
            assert blocked, (idx[k], c[k])
        if not free and not blocked:
            n_pen += 1
            assert c[k] == orc.CLS_TRACE, idx[k]
    assert n_pen > 0                                    # the view shows penumbra
    frac = (c == orc.CLS_TRACE).mean()
    assert 0.0 < frac < 0.25, frac                      # the mask is selective


def test_ray_mask_grows_with_the_cone():
    """A wider cone widens every footprint: the ray mask at a smaller angle
    is contained in the mask at a larger one."""
    s = wl.scene_boxes()
    sc = orc.Scene(s)
    cam = wl.boxes_camera(96, 96)
    m = orc.ShadowMap(sc, LIGHT, 512)
    masks, ok = [], None
    for deg in (0.25, 0.5, 3.0):
        tr = orc.trace_selective(sc, cam, orc.TraceParams(cone_half_angle_deg=[deg]), [m])
        fg = np.isfinite(tr["depth"])
        masks.append(fg & (tr["cls"][:, 0] == orc.CLS_TRACE))
        a = tr["amb_cls"][:, 0] == 0
        ok = a if ok is None else ok & a
    for small, large in zip(masks, masks[1:]):
        assert not (small & ~large & ok).any()
    assert masks[0].sum() < masks[2].sum()


def test_hard_shadows_mask_only_the_boundary():
    """theta = 0: the classification of lit and umbra pixels is the hard
    shadow ray's verdict; the mask is a thin band along shadow edges."""
    s = wl.scene_boxes()
    sc = orc.Scene(s)
    cam = wl.boxes_camera(96, 96)
    m = orc.ShadowMap(sc, LIGHT, 512)
    tr = orc.trace_selective(sc, cam, orc.TraceParams(cone_half_angle_deg=[0.0]), [m])
    fg = np.isfinite(tr["depth"]) & (tr["amb_primary"] == 0) & (tr["amb_shadow"] == 0)
    c = tr["cls"][:, 0]
    ok = fg & (tr["amb_cls"][:, 0] == 0) & (c != orc.CLS_TRACE)
    assert (tr["shadow_mask"][ok] == tr["shadow_mask_full"][ok]).all()
    assert ((c == orc.CLS_TRACE) & fg).mean() < 0.05


def test_two_lights_and_an_untraced_light():
    """Bit k follows light k's own map; a light without a map is traced
    everywhere."""
    s = wl.scene_boxes()
    sc = orc.Scene(s)
    cam = wl.boxes_camera(64, 64)
    l2 = (-0.5, 0.8, 0.1)
    tp = orc.TraceParams(light_dirs=[LIGHT, l2], cone_half_angle_deg=[0.5, 3.0])
    m0 = orc.ShadowMap(sc, LIGHT, 256)
    tr = orc.trace_selective(sc, cam, tp, [m0, None])
    fg = np.isfinite(tr["depth"])
    assert ((tr["traced"][fg] & 2) == 2).all()
    assert ((tr["shadow_mask"] & 2) == (tr["shadow_mask_full"] & 2)).all()
    c0 = tr["cls"][:, 0]
    lit = fg & (c0 == orc.CLS_LIT)
    assert ((tr["shadow_mask"][lit] & 1) == 1).all()
    assert ((tr["traced"][fg & (c0 != orc.CLS_TRACE)] & 1) == 0).all()
