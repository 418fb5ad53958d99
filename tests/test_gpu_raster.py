"""Rasterised primary visibility (DHR_PRIMARY_RASTER, the default) against
the traversed primary rays (DHR_PRIMARY_TRAVERSE): both define the G-buffer
as the closest hit of the pixel-centre ray (ties to the smaller original
triangle index), so every output -- depth/normal bytes, mesh ids, shadow
bits, AO counts -- must be identical, byte for byte.  The oracle parity tests
(test_gpu_trace.py and the rest) run the default, rasterised path.

Cases: both storage forms, ragged and tiny images, the 1080p terrain frames
of the benchmark (the camera flies low over terrain, so triangles cross the
frustum's side planes and are clipped), a camera inside a closed sphere, a
skewed (non-orthonormal) camera basis, images too small for the bins and
lists that overflow their slots (those tiles are traversed), empty and
one-triangle scenes, and the selective trace.
"""
import numpy as np
import pytest

import paper_2406_06963_b300 as dhrs
import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(scene, cam, params, precision=dhrs.DHR_FP32, maps=None):
    g = dhrs.GBuffer(cam.width, cam.height, precision)
    mask = torch.empty((cam.height, cam.width), dtype=torch.uint8, device="cuda")
    ao = torch.empty_like(mask)
    if maps is None:
        dhrs.trace_visibility(scene, cam, params, g, mask, ao)
        rm = None
    else:
        rm = torch.empty_like(mask)
        dhrs.trace_visibility_selective(scene, cam, params, maps, g, mask, ao, rm)
    torch.cuda.synchronize()
    out = dict(dn=g.depth_normal.cpu().numpy().view(np.uint8), mesh=g.mesh.cpu().numpy().view(np.uint8),
               mask=mask.cpu().numpy(), ao=ao.cpu().numpy())
    if rm is not None:
        out["ray_mask"] = rm.cpu().numpy()
    return out


def _same(scene, cam, precision=dhrs.DHR_FP32, maps=None, **kw):
    r = _run(scene, cam, dhrs.TraceParams(primary=dhrs.PRIMARY_RASTER, **kw), precision, maps)
    t = _run(scene, cam, dhrs.TraceParams(primary=dhrs.PRIMARY_TRAVERSE, **kw), precision, maps)
    for k in r:
        assert np.array_equal(r[k], t[k]), (k, int((r[k] != t[k]).sum()))
    return r


@pytest.fixture(scope="module")
def boxes():
    return dhrs.Scene(wl.scene_boxes())


@pytest.mark.parametrize("precision", [dhrs.DHR_FP32, dhrs.DHR_FP16])
def test_boxes_views(boxes, precision):
    for cam in [wl.boxes_camera(256, 256), wl.look_at((0.3, 0.6, 2.0), (0.0, 0.2, -4.0), 320, 200),
                wl.look_at((0.0, 12.0, 0.01), (0.0, 0.0, 0.0), 128, 128)]:
        out = _same(boxes, cam, precision, ao_spp=2, frame=3)
        assert (out["mesh"].view(np.uint32) != 0xFFFFFFFF).any()


@pytest.mark.parametrize("w,h", [(37, 23), (1, 1), (17, 129), (300, 7), (2, 1)])
def test_ragged_sizes(boxes, w, h):
    _same(boxes, wl.look_at((1.0, 5.0, 9.0), (0.0, 0.5, 0.0), w, h), frame=1)


def test_small_images_and_list_overflow(boxes):
    """Close-ups at 15 x 15 (no room for the lists in the mesh-id buffer:
    traversed), 16 x 16, 24 x 20 and 40 x 32; terrain776k at 64 x 36: about
    10^5 (tile, triangle) pairs for about 2,100 list slots, so the tiles whose
    lists do not fit are traversed."""
    for w, h in ((15, 15), (16, 16), (24, 20), (40, 32)):
        _same(boxes, wl.look_at((0.5, 1.0, 2.5), (0.0, 0.5, 0.0), w, h, fov_y_deg=100.0), frame=2)
    s = wl.scene_terrain()
    _same(dhrs.Scene(s), wl.spline_path(s["terrain"], 60, 64, 36)[10], frame=10)


def test_screen_filling_triangles(boxes):
    """A close-up at 512 x 256 (4,096 tiles): the ground's two triangles each
    cover more than one 1,024-tile piece of the big list, the boxes' faces
    fall in the medium list (33-256 tiles) and in the threads' own range."""
    cam = wl.look_at((0.5, 1.0, 2.5), (0.0, 0.5, 0.0), 512, 256, fov_y_deg=100.0)
    out = _same(boxes, cam, frame=2)
    assert (out["mesh"].view(np.uint32) != 0xFFFFFFFF).mean() > 0.5


def test_camera_inside_closed_sphere():
    s = dhrs.Scene(wl.scene_enclosing_sphere())
    cam = wl.look_at((0.0, 0.0, 0.0), (1.0, 0.2, 0.3), 96, 64)
    out = _same(s, cam)
    assert (out["mesh"].view(np.uint32) != 0xFFFFFFFF).all()


def test_skewed_camera_basis(boxes):
    """right and up neither unit nor orthogonal to forward: the rays are
    still forward + sx right + sy up, and the rasteriser inverts the basis."""
    cam = wl.boxes_camera(160, 120)
    f = np.asarray(cam.forward, np.float64)
    cam.right = tuple((np.asarray(cam.right) * 1.3 + 0.2 * f).tolist())
    cam.up = tuple((np.asarray(cam.up) * 0.8 + 0.1 * np.asarray(cam.right)).tolist())
    _same(boxes, cam, frame=4)


def test_terrain_1080p_frames():
    s = wl.scene_terrain()
    sc = dhrs.Scene(s)
    cams = wl.spline_path(s["terrain"], 60, 1920, 1080)
    for f in (0, 19, 47):
        _same(sc, cams[f], frame=f)
    _same(sc, cams[5], dhrs.DHR_FP16, frame=5)


def test_selective_trace_both_primaries():
    s = wl.scene_terrain(n_spheres=20, n_boxes=10, terrain_n=24)
    sc = dhrs.Scene(s)
    cam = wl.spline_path(s["terrain"], 8, 320, 180)[2]
    _same(sc, cam, maps=[dhrs.ShadowMap(sc, (0.3, 1.0, 0.2), 512)], frame=2)


def test_empty_and_single_triangle_scenes():
    empty = dict(vertices=np.zeros((0, 3), np.float32), indices=np.zeros((0, 3), np.uint32),
                 mesh_ids=np.zeros(0, np.uint32))
    cam = wl.look_at((0, 2, 3), (0, 0, 0), 40, 30)
    out = _same(dhrs.Scene(empty), cam, ao_spp=3)
    assert (out["mesh"].view(np.uint32) == 0xFFFFFFFF).all()
    q = wl.scene_quad([[-1, 0, -1], [-1, 0, 1], [1, 0, 1], [1, 0, -1]], 9)
    one = dict(vertices=q["vertices"], indices=q["indices"][:1], mesh_ids=q["mesh_ids"][:1])
    out = _same(dhrs.Scene(one), cam, ao_spp=2)
    assert (out["mesh"].view(np.uint32) == 9).any()


def test_bad_primary_mode_rejected(boxes):
    cam = wl.boxes_camera(16, 16)
    with pytest.raises(dhrs.DhrError) as e:
        _run(boxes, cam, dhrs.TraceParams(primary=2))
    assert e.value.status == 1


def test_trace_timed_outputs_and_parts(boxes):
    """dhr_trace_timed: the same outputs as dhr_trace_visibility, and the two
    device times (primary pre-pass ~0 when traversed)."""
    cam = wl.boxes_camera(200, 150)
    ref = _run(boxes, cam, dhrs.TraceParams(frame=6))
    g = dhrs.GBuffer(200, 150)
    mask = torch.empty((150, 200), dtype=torch.uint8, device="cuda")
    ao = torch.empty_like(mask)
    pre, ker = dhrs.trace_timed(boxes, cam, dhrs.TraceParams(frame=6), g, mask, ao)
    assert pre > 0.0 and ker > 0.0
    assert np.array_equal(g.depth_normal.cpu().numpy().view(np.uint8), ref["dn"])
    assert np.array_equal(mask.cpu().numpy(), ref["mask"]) and np.array_equal(ao.cpu().numpy(), ref["ao"])
    pre_t, ker_t = dhrs.trace_timed(boxes, cam, dhrs.TraceParams(frame=6, primary=dhrs.PRIMARY_TRAVERSE), g, mask, ao)
    assert 0.0 <= pre_t < 0.05 and ker_t > 0.0
