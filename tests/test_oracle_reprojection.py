"""Pins of the oracle's temporal reprojection (Section 3.3: back-project the
pixel's world position into the previous frame and discard history samples
inconsistent in projected depth, normal or mesh id).

The depth test is |z_prev(q) - z'| <= 0.01 z' + 2 max(|dz/dx|, |dz/dy|),
with dz/dx, dz/dy the one-sided screen-space depth differences of smaller
magnitude.  The G-buffers here are written from closed forms (a floor seen
at grazing angles by a level camera, fronto-parallel planes with a depth
step), and every expected value -- the previous-frame pixel position, the
bilinear weights, the depth slope of a row -- is computed in double from
that geometry, not by the oracle:

* a one-pixel bilinear tap on a grazing floor stays valid because of the
  slope term (without it the tap is rejected and the blend renormalises);
* a history depth offset of 1.5 slopes (beyond the 1 %) is accepted and
  one of 2.5 slopes is rejected, which brackets the factor 2 (on the convex
  floor the far-side difference is up to 1.4 times the near-side one, so
  this also fixes which side is taken);
* beside a depth step one difference is 0, and on a one-pixel ridge the two
  differ in sign: the slope is 0 (minmod) and a 2 % depth change is
  rejected there as on any flat surface;
* the binary32 decision the temporal step takes equals the plain double
  definition on every pixel not within a stated margin of a threshold.
"""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl

W, H = 48, 40
CAM_H = 1.0


def _floor_cam(height):
    return wl.look_at((0.0, height, 0.0), (0.0, height, -1.0), W, H)


def _sy(cam, rows):
    """Vertical screen coordinate of pixel-centre rows (double)."""
    t = float(np.float32(cam.tan_half_fov_y))
    return (1.0 - 2.0 * (np.asarray(rows, np.float64) + 0.5) / H) * t


def _floor_depth(cam, height, rows):
    """Linear depth of the floor y = 0 seen from `height` (+inf above the
    horizon): the ray f + sx r + sy u meets it at depth height / -sy."""
    sy = _sy(cam, rows)
    with np.errstate(divide="ignore"):
        return np.where(sy < 0, height / -np.minimum(sy, -1e-300), np.inf)


def _floor_gbuffer(cam, height):
    z = _floor_depth(cam, height, np.arange(H)).astype(np.float32)
    zn = np.zeros((H, W, 4), np.float32)
    zn[..., 0] = z[:, None]
    fg = np.isfinite(z)[:, None] & np.ones((1, W), bool)
    zn[fg, 1:] = (0.0, 1.0, 0.0)
    mesh = np.where(fg, 0, 0xFFFFFFFF).astype(np.uint32)
    return zn, mesh


def _row_slope(cam, height, y):
    """Smaller of the two one-sided depth differences of row y (double)."""
    z = _floor_depth(cam, height, [y - 1, y, y + 1])
    d = [abs(z[1] - z[0]) if np.isfinite(z[0]) else np.inf, abs(z[2] - z[1]) if y + 1 < H else np.inf]
    return min(d)


# rows whose screen-space depth gradient is steep (5-25 % of the depth per
# pixel) but whose far-side tap stays within two near-side slopes
ROWS = np.arange(26, 40)


def test_grazing_floor_keeps_one_pixel_taps():
    """The camera rises by 0.05: every floor point moves |sy|/t pixels down
    the screen (0.3-1 px on ROWS).  The history at the back-projected
    position is the bilinear blend of the two rows around it; both rows
    must be kept although their depths differ from z' by up to 20 %."""
    cam, camp = _floor_cam(CAM_H), _floor_cam(CAM_H + 0.05)
    zn, mesh = _floor_gbuffer(cam, CAM_H)
    znp, meshp = _floor_gbuffer(camp, CAM_H + 0.05)
    mu_row = (np.arange(H) * 0.37) % 1.0
    mom = np.zeros((H, W, 4))
    mom[..., 0] = mu_row[:, None]
    s = 0.25
    ao = np.full((H, W), round(s * 255), np.uint8)
    res = orc.svgf_temporal(zn, mesh, cam, np.zeros((H, W), np.uint8), ao, orc.SvgfParams(ao_spp=255),
                            prev=(znp, meshp, camp), mom=mom, hist=np.ones((H, W), np.int32))
    t = float(np.float32(cam.tan_half_fov_y))
    slope_used = used = 0
    for y in ROWS:
        sy = _sy(cam, [y])[0]
        z = _floor_depth(cam, CAM_H, [y])[0]
        # previous-frame position: the point keeps its depth z' = z and its
        # vertical screen coordinate scales with the camera height
        v = (1.0 - (sy / t) * (CAM_H + 0.05) / CAM_H) * 0.5 * H - 0.5
        r0 = int(math.floor(v))
        f = v - r0
        if not (0.05 < f < 0.95 and r0 + 1 < H):
            continue                # one tap carries (almost) all the weight
        used += 1
        zt = _floor_depth(camp, CAM_H + 0.05, [r0, r0 + 1])
        dz = np.abs(zt - z)
        lim = 0.01 * z + 2.0 * _row_slope(cam, CAM_H, y)
        assert (dz <= 0.9 * lim).all(), (y, dz, lim)
        slope_used += int((dz > 0.011 * z).any())
        expect = (1 - f) * mu_row[r0] + f * mu_row[r0 + 1]
        expect += 0.5 * (round(s * 255) / 255 - expect)        # n = 2: alpha_eff = 1/2
        assert (res["hist"][y] == 2).all()
        assert np.allclose(res["mom"][y, :, 0], expect, atol=1e-4), (y, res["mom"][y, 0, 0], expect)
    # every row checked needs the slope term for at least one of its taps
    assert used >= 10 and slope_used == used


@pytest.mark.parametrize("k,valid", [(1.5, True), (2.5, False)])
def test_depth_tolerance_is_two_slopes(k, valid):
    """Static camera; the history's depth is 1 % + k slopes behind the
    current one: accepted for k = 1.5, rejected for k = 2.5."""
    cam = _floor_cam(CAM_H)
    zn, mesh = _floor_gbuffer(cam, CAM_H)
    znp = zn.copy()
    for y in ROWS:
        z = _floor_depth(cam, CAM_H, [y])[0]
        znp[y, :, 0] = np.float32(1.01 * z + k * _row_slope(cam, CAM_H, y))
    res = orc.svgf_temporal(zn, mesh, cam, np.zeros((H, W), np.uint8), np.zeros((H, W), np.uint8),
                            orc.SvgfParams(ao_spp=255), prev=(znp, mesh, cam), hist=np.full((H, W), 6, np.int32))
    assert (res["valid"][ROWS] == int(valid)).all()
    assert (res["hist"][ROWS] == (7 if valid else 1)).all()


@pytest.mark.parametrize("scale,valid", [(1.02, False), (1.005, True)])
def test_depth_step_takes_the_smaller_side(scale, valid):
    """Fronto-parallel planes at depths 8 (x < 20) and 80 (x >= 20) of one
    mesh.  Beside the step one neighbour differs by 72, the other by 0: the
    slope is 0 and the tolerance stays 1 % there too."""
    cam = wl.look_at((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), W, H)
    zn = np.zeros((H, W, 4), np.float32)
    zn[..., 0] = np.where(np.arange(W) < 20, 8.0, 80.0)[None, :]
    zn[..., 3] = 1.0
    mesh = np.zeros((H, W), np.uint32)
    znp = zn.copy()
    znp[..., 0] *= np.float32(scale)
    res = orc.svgf_temporal(zn, mesh, cam, np.zeros((H, W), np.uint8), np.zeros((H, W), np.uint8),
                            orc.SvgfParams(ao_spp=255), prev=(znp, mesh, cam), hist=np.full((H, W), 3, np.int32))
    assert (res["valid"] == int(valid)).all(), np.argwhere(res["valid"] != int(valid))[:5]


# margins within which binary32 and double may decide differently: the
# projected position (pixels), the depth test (relative), the normal cosine
# and the valid weight sum
TOL = dict(px=1e-3, z=1e-5, n=1e-5, w=1e-6)


def _compare(zn, mesh, cam, prev):
    d32, d64, m = orc.reproject_check(zn, mesh, cam, prev)
    near = (m[..., 0] < TOL["px"]) | (m[..., 1] < TOL["z"]) | (m[..., 2] < TOL["n"]) | (m[..., 3] < TOL["w"])
    fg = mesh != 0xFFFFFFFF
    diff = (d32 != d64).any(-1)
    return dict(fg=int(fg.sum()), valid=int(d64[..., 0][fg].sum()), near=int((near & fg).sum()),
                bad=int((diff & ~near).sum()), differ=int(diff.sum()))


def _boxes_and_spheres():
    """The box scene plus three level-2 icospheres (curved surfaces)."""
    v, t = wl.icosphere(2)
    parts = [wl.scene_boxes()]
    for k, (c, r) in enumerate((((0.0, 1.0, 0.0), 1.0), ((1.8, 0.6, 1.2), 0.6), ((-1.5, 0.8, 0.8), 0.8))):
        parts.append(dict(vertices=(v * r + np.array(c)).astype(np.float32), indices=t.astype(np.uint32),
                          mesh_ids=np.full(len(t), 100 + k, np.uint32)))
    return wl.merge(*parts)


def _frames_boxes(scene, cams):
    S = orc.Scene(scene)
    out = []
    for f, c in enumerate(cams):
        tr = orc.trace(S, c, orc.TraceParams(frame=f))
        out.append(orc.gbuffer_f32(tr, c.width, c.height))
    return out


@pytest.mark.parametrize("name", ["boxes", "spheres"])
def test_binary32_decision_equals_double_definition(name):
    """Moving cameras over the box scene (flat faces, depth steps) and the
    box scene with icospheres (curved surfaces): the two decisions agree on
    every pixel whose double decision is not within TOL of flipping."""
    scene = wl.scene_boxes() if name == "boxes" else _boxes_and_spheres()
    cams = wl.orbit_path(3, 96, 80, degrees=6.0)
    frames = _frames_boxes(scene, cams)
    tot = dict(fg=0, valid=0, near=0, bad=0, differ=0)
    for f in (1, 2):
        r = _compare(*frames[f], cams[f], (*frames[f - 1], cams[f - 1]))
        tot = {k: tot[k] + r[k] for k in tot}
    assert tot["bad"] == 0, tot
    assert tot["valid"] > 0.8 * tot["fg"], tot
    assert tot["near"] < 0.02 * tot["fg"], tot


def test_binary32_decision_equals_double_definition_grazing():
    """The grazing floor with a camera that moves forward and rises (depth
    slopes of 5-200 % per pixel)."""
    cam = _floor_cam(CAM_H)
    camp = wl.look_at((0.0, CAM_H - 0.03, 0.21), (0.0, CAM_H - 0.03, -0.79), W, H)
    zn, mesh = _floor_gbuffer(cam, CAM_H)
    znp, meshp = _floor_gbuffer(camp, CAM_H - 0.03)
    r = _compare(zn, mesh, cam, (znp, meshp, camp))
    assert r["bad"] == 0, r
    assert r["valid"] > 0.5 * r["fg"], r


def test_ridge_slope_is_zero():
    """A one-pixel column 0.5 in front of a fronto-parallel plane at depth 8:
    its two horizontal one-sided depth differences are +0.5 and -0.5, so its
    slope is 0 (minmod) and a 2 % depth change of its history is rejected
    as anywhere on a flat surface, while a 0.5 % change is kept."""
    cam = wl.look_at((0.0, 0.0, 0.0), (0.0, 0.0, -1.0), W, H)
    zn = np.zeros((H, W, 4), np.float32)
    zn[..., 0] = 8.0
    zn[:, 20, 0] = 7.5
    zn[..., 3] = 1.0
    mesh = np.zeros((H, W), np.uint32)
    for scale, valid in ((1.02, 0), (1.005, 1)):
        znp = zn.copy()
        znp[..., 0] *= np.float32(scale)
        res = orc.svgf_temporal(zn, mesh, cam, np.zeros((H, W), np.uint8), np.zeros((H, W), np.uint8),
                                orc.SvgfParams(ao_spp=255), prev=(znp, mesh, cam), hist=np.full((H, W), 3, np.int32))
        assert (res["valid"][:, 20] == valid).all(), scale
