"""Pins for the oracle's delay reprojection (Section 4.1, Fig. 5)."""
import numpy as np

import oracle as orc
import workloads as wl


def _plane(cam):
    S = orc.Scene(wl.scene_quad([[-50, -50, -8], [50, -50, -8], [50, 50, -8], [-50, 50, -8]], 3))
    tr = orc.trace(S, cam, orc.TraceParams())
    return orc.gbuffer_f32(tr, cam.width, cam.height)


def test_warp_identity_pose_copies_exactly():
    s = wl.scene_boxes()
    S = orc.Scene(s)
    cam = wl.boxes_camera(64, 48)
    zn, mesh = orc.gbuffer_f32(orc.trace(S, cam, orc.TraceParams()), 64, 48)
    r = np.random.default_rng(0)
    a, b = r.random((48, 64)), r.random((48, 64))
    oa, ob, valid = orc.delay_warp(zn, mesh, cam, zn, mesh, cam, a, b)
    fg = np.isfinite(zn[..., 0])
    assert (valid == fg).all()
    assert np.array_equal(oa[fg], a[fg]) and np.array_equal(ob[fg], b[fg])
    assert (oa[~fg] == 1).all()


def test_warp_follows_camera_shift():
    """Target camera moved sideways by exactly 2 pixels over a fronto-parallel
    plane: target pixel x shows source pixel x + 2; pixels whose source is off
    screen fall back to 1."""
    W, H = 40, 30
    cam_s = wl.look_at((0, 0, 0), (0, 0, -1), W, H)
    dx = 2 * 2.0 * 8.0 * cam_s.tan_half_fov_y * (W / H) / W
    cam_t = wl.look_at((dx, 0, 0), (dx, 0, -1), W, H)
    zs, ms = _plane(cam_s)
    zt, mt = _plane(cam_t)
    src = np.random.default_rng(1).random((H, W))
    oa, _, valid = orc.delay_warp(zt, mt, cam_t, zs, ms, cam_s, src, src)
    assert (valid[:, :W - 2] == 1).all() and (valid[:, W - 1:] == 0).all()
    assert np.array_equal(oa[:, :W - 2], src[:, 2:])
    assert (oa[:, W - 1:] == 1).all()


def test_warp_rejects_other_surfaces():
    """A source of another mesh id (an occluder that moved away) is not used."""
    W, H = 32, 24
    cam = wl.look_at((0, 0, 0), (0, 0, -1), W, H)
    zt, mt = _plane(cam)
    zs, ms = zt.copy(), mt.copy() + 1
    oa, ob, valid = orc.delay_warp(zt, mt, cam, zs, ms, cam, np.zeros((H, W)), np.zeros((H, W)))
    assert (valid == 0).all() and (oa == 1).all() and (ob == 1).all()
