"""GPU parity of the selective shadow rays (Section 5: the shadow-map ray
mask) against the oracle.

* Shadow map: every texel against the oracle's brute-force texel rays
  (boxes194 at 256^2, a small terrain at 256^2); at the full size
  (terrain776k, 4096^2) on sampled texels, and the pyramid levels by their
  definition (minimum of 2 x 2 texels of the level below).
* Classification: every pixel's class (lit / umbra / ray) equals the
  oracle's wherever the oracle does not flag a decision as within its
  margin; the shadow bit of a called ray follows the ray parity bar.
* Full size (terrain776k, 1920x1080): G-buffer and AO are those of the full
  trace byte for byte, every called ray gives the full trace's bit, and the
  shadow map's verdicts disagree with the full trace's rays on few pixels.
"""
import numpy as np
import pytest

import oracle as orc
import paper_2406_06963_b300 as dhrs
import workloads as wl
from gpu_util import compare_trace, gpu_params, trace_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LIGHT = (0.3, 1.0, 0.2)


def _check_map(g_map, o_map):
    info = g_map.info()
    f = o_map.frame_dict()
    assert info["resolution"] == f["res"]
    for a, b in (("light_dir", "L"), ("axis_u", "eu"), ("axis_v", "ev")):
        assert np.allclose(info[a], f[b], atol=1e-7)
    for a, b in (("u0", "u0"), ("v0", "v0"), ("texel", "w"), ("plane", "h")):
        assert abs(info[a] - f[b]) <= 1e-6 * max(1.0, abs(f[b]))
    S = g_map.depth().cpu().numpy().astype(np.float64)
    ok = o_map.amb == 0
    gi, oi = np.isinf(S), np.isinf(o_map.depth)
    assert not (ok & (gi != oi)).any(), int((ok & (gi != oi)).sum())
    both = ok & ~gi & ~oi
    err = np.abs(S[both] - o_map.depth[both])
    assert (err <= _depth_tol(f, o_map.depth[both])).all(), err.max(initial=0.0)
    assert info["depth_min"] == np.float32(S.min())
    return S


def _depth_tol(f, d):
    """The kernel builds each texel ray's origin in binary32 from coordinates
    of magnitude up to |h| + |u0| + |v0| + R w: a few units in the last
    place of those, plus the depth's own rounding."""
    scale = abs(f["h"]) + abs(f["u0"]) + abs(f["v0"]) + f["res"] * f["w"]
    return 1e-6 * (scale + np.abs(d))


def _pyramid_ok(g_map):
    info = g_map.info()
    R, L = info["resolution"], info["levels"]
    n = (4 * R * R - 1) // 3           # sum of (R >> l)^2 over all levels
    allv = torch.as_tensor(dhrs._DevArray(info["depth"], (n,), "<f4"), device="cuda").clone()
    off = 0
    prev = None
    for lv in range(L):
        r = R >> lv
        cur = allv[off:off + r * r].view(r, r)
        if prev is not None:
            want = torch.minimum(torch.minimum(prev[0::2, 0::2], prev[0::2, 1::2]),
                                 torch.minimum(prev[1::2, 0::2], prev[1::2, 1::2]))
            assert torch.equal(cur, want), lv
        prev = cur
        off += r * r
    assert off == n


@pytest.fixture(scope="module")
def boxes():
    s = wl.scene_boxes()
    return s, dhrs.Scene(s), orc.Scene(s)


def test_shadow_map_matches_oracle_boxes(boxes):
    s, g, o = boxes
    for light in (LIGHT, (0.0, 1.0, 0.0), (-0.5, 0.8, 0.1)):
        gm = dhrs.ShadowMap(g, light, 256)
        om = orc.ShadowMap(o, light, 256)
        _check_map(gm, om)
        _pyramid_ok(gm)


def test_shadow_map_matches_oracle_small_terrain():
    s = wl.scene_terrain(n_spheres=20, n_boxes=10, terrain_n=24)
    gm = dhrs.ShadowMap(dhrs.Scene(s), LIGHT, 256)
    om = orc.ShadowMap(orc.Scene(s), LIGHT, 256)
    _check_map(gm, om)


def test_shadow_map_terrain_full_size_sampled():
    """terrain776k at 4096^2 (the selective bench configuration): 512
    seeded texels against the oracle, and every pyramid level."""
    s = wl.scene_terrain()
    g = dhrs.Scene(s)
    gm = dhrs.ShadowMap(g, LIGHT, 4096)
    info = gm.info()
    assert info["resolution"] == 4096 and info["levels"] == 13
    om = orc.ShadowMap(orc.Scene(s), LIGHT, 4096, full=False)
    r = np.random.default_rng(3)
    ij = r.integers(0, 4096, (512, 2))
    d, amb = om.texels(ij)
    S = gm.depth().cpu().numpy().astype(np.float64)
    gv = S[ij[:, 1], ij[:, 0]]
    ok = amb == 0
    assert not (ok & (np.isinf(gv) != np.isinf(d))).any()
    both = ok & np.isfinite(gv) & np.isfinite(d)
    assert both.sum() > 400
    assert (np.abs(gv[both] - d[both]) <= _depth_tol(om.frame_dict(), d[both])).all()
    _pyramid_ok(gm)


def _selective_gpu(scene, cam, params, maps, precision=dhrs.DHR_FP32):
    g = dhrs.GBuffer(cam.width, cam.height, precision)
    mask = torch.empty((cam.height, cam.width), dtype=torch.uint8, device="cuda")
    ao = torch.empty_like(mask)
    rm = torch.full_like(mask, 0xEE)
    dhrs.trace_visibility_selective(scene, cam, params, maps, g, mask, ao, rm)
    torch.cuda.synchronize()
    zn = g.to_fp32().depth_normal.cpu().numpy().reshape(-1, 4)
    return dict(depth=zn[:, 0].astype(np.float64), normal=zn[:, 1:].astype(np.float64),
                mesh=g.mesh_u32().ravel(), shadow_mask=mask.cpu().numpy().ravel(),
                ao_count=ao.cpu().numpy().ravel(), ray_mask=rm.cpu().numpy().ravel())


def _gpu_classes(gpu, k):
    traced = (gpu["ray_mask"] >> k) & 1
    bit = (gpu["shadow_mask"] >> k) & 1
    return np.where(traced == 1, orc.CLS_TRACE, np.where(bit == 1, orc.CLS_LIT, orc.CLS_UMBRA))


@pytest.mark.parametrize("deg,precision", [(0.5, dhrs.DHR_FP32), (3.0, dhrs.DHR_FP32), (0.5, dhrs.DHR_FP16),
                                           (0.0, dhrs.DHR_FP32)])
def test_selective_trace_matches_oracle_boxes(boxes, deg, precision):
    s, g, o = boxes
    W, H = 192, 160
    cam = wl.look_at((2.0, 7.0, 9.0), (0.0, 0.3, 0.0), W, H)
    tp = orc.TraceParams(cone_half_angle_deg=[deg], ao_spp=2, frame=5)
    om = orc.ShadowMap(o, LIGHT, 512)
    gm = dhrs.ShadowMap(g, LIGHT, 512)
    ref = orc.trace_selective(o, cam, tp, [om])
    gpu = _selective_gpu(g, cam, gpu_params(tp), [gm], precision)
    fg = ref["mesh"] != 0xFFFFFFFF
    sure = fg & (ref["amb_primary"] == 0) & (ref["amb_cls"][:, 0] == 0) & (gpu["mesh"] == ref["mesh"])
    gc = _gpu_classes(gpu, 0)
    bad = sure & (gc != ref["cls"][:, 0])
    assert not bad.any(), (int(bad.sum()), np.nonzero(bad)[0][:10])
    assert (gpu["ray_mask"][~fg & (gpu["mesh"] == 0xFFFFFFFF)] == 0).all()
    # the rest of the trace (G-buffer, AO, bits of called rays) at the ray bar
    r2 = dict(ref)
    r2["amb_shadow"] = ref["amb_shadow"] | ref["amb_cls"][:, 0]
    res = compare_trace(gpu, r2, np.arange(W * H), 1, 2)
    assert res["primary_unexplained"] == 0 and res["shadow_unexplained"] == 0, res
    assert res["ao_unexplained"] == 0 and res["disagree_frac"] <= 1e-3, res
    frac = (gc[fg] == orc.CLS_TRACE).mean()
    assert frac < 0.3, frac


def test_selective_two_lights_one_without_map(boxes):
    s, g, o = boxes
    cam = wl.boxes_camera(128, 128)
    l2 = (-0.5, 0.8, 0.1)
    tp = orc.TraceParams(light_dirs=[LIGHT, l2], cone_half_angle_deg=[0.5, 3.0], frame=2)
    ref = orc.trace_selective(o, cam, tp, [orc.ShadowMap(o, LIGHT, 256), None])
    gpu = _selective_gpu(g, cam, gpu_params(tp), [dhrs.ShadowMap(g, LIGHT, 256), None])
    fg = (ref["mesh"] != 0xFFFFFFFF) & (gpu["mesh"] == ref["mesh"])
    assert ((gpu["ray_mask"][fg] & 2) == 2).all()
    sure = fg & (ref["amb_primary"] == 0) & (ref["amb_cls"][:, 0] == 0)
    assert (_gpu_classes(gpu, 0)[sure] == ref["cls"][sure, 0]).all()
    r2 = dict(ref)
    r2["amb_shadow"] = ref["amb_shadow"] | ref["amb_cls"][:, 0]
    res = compare_trace(gpu, r2, np.arange(128 * 128), 2, 1)
    assert res["shadow_unexplained"] == 0 and res["primary_unexplained"] == 0, res


def test_selective_small_terrain_matches_oracle():
    s = wl.scene_terrain(n_spheres=20, n_boxes=10, terrain_n=24)
    g, o = dhrs.Scene(s), orc.Scene(s)
    cams = wl.spline_path(s["terrain"], 8, 160, 96)
    tp = orc.TraceParams(frame=1)
    ref = orc.trace_selective(o, cams[3], tp, [orc.ShadowMap(o, LIGHT, 256)])
    gpu = _selective_gpu(g, cams[3], gpu_params(tp), [dhrs.ShadowMap(g, LIGHT, 256)])
    fg = (ref["mesh"] != 0xFFFFFFFF) & (gpu["mesh"] == ref["mesh"])
    sure = fg & (ref["amb_primary"] == 0) & (ref["amb_cls"][:, 0] == 0)
    assert sure.sum() > 0.8 * fg.sum()
    assert (_gpu_classes(gpu, 0)[sure] == ref["cls"][sure, 0]).all()


def test_selective_terrain_1080p_against_full_trace():
    """1920x1080, terrain776k, 4096^2 map: the selective trace changes
    nothing but the shadow bits of uncalled rays, and those agree with the
    full trace's rays on all but a few pixels."""
    s = wl.scene_terrain()
    g = dhrs.Scene(s)
    gm = dhrs.ShadowMap(g, LIGHT, 4096)
    cams = wl.spline_path(s["terrain"], 60, 1920, 1080)
    for f in (0, 41):
        p = dhrs.TraceParams(frame=f)
        full = trace_gpu(g, cams[f], p)
        sel = _selective_gpu(g, cams[f], p, [gm])
        for k in ("depth", "normal", "mesh", "ao_count"):
            assert np.array_equal(full[k], sel[k]), k
        fg = full["mesh"] != 0xFFFFFFFF
        called = (sel["ray_mask"] & 1) == 1
        assert not (called & ~fg).any()
        assert np.array_equal(full["shadow_mask"][called], sel["shadow_mask"][called])
        diff = fg & ~called & (full["shadow_mask"] != sel["shadow_mask"])
        frac_called = called[fg].mean()
        assert frac_called < 0.5, frac_called
        assert diff.sum() <= 1e-3 * fg.sum(), (int(diff.sum()), int(fg.sum()))


def test_selective_rejects_bad_maps_and_arguments(boxes):
    s, g, o = boxes
    cam = wl.boxes_camera(32, 32)
    gb = dhrs.GBuffer(32, 32)
    m = torch.empty((32, 32), dtype=torch.uint8, device="cuda")
    a = torch.empty_like(m)
    other = dhrs.Scene(wl.scene_boxes(index=3))
    for bad_map in (dhrs.ShadowMap(other, LIGHT, 64), dhrs.ShadowMap(g, (0.0, 1.0, 0.0), 64)):
        with pytest.raises(dhrs.DhrError) as e:
            dhrs.trace_visibility_selective(g, cam, dhrs.TraceParams(), [bad_map], gb, m, a)
        assert e.value.status == 1
    for res in (8, 100, 16384):
        with pytest.raises(dhrs.DhrError):
            dhrs.ShadowMap(g, LIGHT, res)
    with pytest.raises(dhrs.DhrError):
        dhrs.ShadowMap(g, (0.0, 0.0, 0.0), 64)


def test_selective_empty_scene():
    empty = dict(vertices=np.zeros((0, 3), np.float32), indices=np.zeros((0, 3), np.uint32),
                 mesh_ids=np.zeros(0, np.uint32))
    g = dhrs.Scene(empty)
    gm = dhrs.ShadowMap(g, LIGHT, 16)
    assert np.isinf(gm.depth().cpu().numpy()).all() and np.isinf(gm.info()["depth_min"])
    gpu = _selective_gpu(g, wl.look_at((0, 2, 3), (0, 0, 0), 20, 10), dhrs.TraceParams(ao_spp=3), [gm])
    assert (gpu["mesh"] == 0xFFFFFFFF).all() and (gpu["ray_mask"] == 0).all()
    assert (gpu["shadow_mask"] == 1).all() and (gpu["ao_count"] == 3).all()
