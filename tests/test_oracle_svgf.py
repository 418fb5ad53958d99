"""Pins for the oracle's modified SVGF (Section 3.3).

Expected values come from closed forms (geometric EMA convergence, running
means, B3-spline kernel sums), from scipy.ndimage normalised convolutions
(an independent routine for the textbook a-trous transform), and from numpy
variances of the same samples.
"""
import math

import numpy as np
import pytest
from scipy import ndimage

import workloads as wl

B3 = np.array([1 / 16, 1 / 4, 3 / 8, 1 / 4, 1 / 16])


def _flat_gbuffer(H, W, depth=5.0, normal=(0.0, 0.0, 1.0), background=None):
    zn = np.zeros((H, W, 4), np.float32)
    zn[..., 0] = depth
    zn[..., 1:] = normal
    mesh = np.zeros((H, W), np.uint32)
    if background is not None:
        zn[background, 0] = np.inf
        zn[background, 1:] = 0
        mesh[background] = 0xFFFFFFFF
    return zn, mesh


K3 = np.array([1 / 4, 1 / 2, 1 / 4])


def _dilated(step, taps=B3):
    k = np.zeros((len(taps) - 1) * step + 1)
    k[::step] = taps
    return np.outer(k, k)


def _normconv(img, mask, kern):
    num = ndimage.correlate(img * mask, kern, mode="constant", cval=0.0)
    den = ndimage.correlate(mask.astype(float), kern, mode="constant", cval=0.0)
    return num / np.where(den > 0, den, 1)


P_TEXTBOOK = dict(sigma_n=0.0, sigma_l=1e30)


def test_atrous_constant_image(orc):
    """A constant colour is a fixed point of every edge-stopping a-trous
    pass, whatever the G-buffer, weights or variance."""
    r = np.random.default_rng(3)
    H, W = 40, 52
    zn = np.zeros((H, W, 4), np.float32)
    zn[..., 0] = r.uniform(1, 50, (H, W))
    n = r.normal(size=(H, W, 3))
    zn[..., 1:] = n / np.linalg.norm(n, axis=-1, keepdims=True)
    bg = r.random((H, W)) < 0.1
    zn[bg, 0] = np.inf
    illum = np.zeros((H, W, 4))
    illum[..., 0] = 0.37
    illum[..., 1] = 0.81
    illum[..., 2:] = r.uniform(0, 0.3, (H, W, 2))
    for step in (1, 2, 4, 8, 16):
        for width in (5, 3):
            out = orc.svgf_atrous(zn, illum, step, orc.SvgfParams(kernel_width=width))
            assert np.allclose(out[~bg, 0], 0.37, atol=1e-12)
            assert np.allclose(out[~bg, 1], 0.81, atol=1e-12)
            assert np.all(out[bg, :2] == 1.0)


@pytest.mark.parametrize("width", [5, 3])
@pytest.mark.parametrize("step", [1, 2, 4, 8, 16])
def test_atrous_reduces_to_textbook_b3(orc, step, width):
    """Without edge stopping (flat depth, sigma_n = 0, sigma_l -> inf) the pass
    is the textbook a-trous transform with holes at `step` -- B3-spline taps,
    or (1/4, 1/2, 1/4) for the smaller kernel of the lightweight denoiser
    (Section 3.3) -- renormalised over in-image foreground taps; variance is
    filtered with the squared kernel."""
    r = np.random.default_rng(step)
    H, W = 48, 70
    bg = r.random((H, W)) < 0.08
    zn, _ = _flat_gbuffer(H, W, background=bg)
    illum = r.uniform(0.05, 1, (H, W, 4))
    out = orc.svgf_atrous(zn, illum, step, orc.SvgfParams(kernel_width=width, **P_TEXTBOOK))
    m = (~bg).astype(float)
    k = _dilated(step, B3 if width == 5 else K3)
    for ch in range(2):
        ref_c = _normconv(illum[..., ch], m, k)
        num_v = ndimage.correlate(illum[..., 2 + ch] * m, k * k, mode="constant")
        den = ndimage.correlate(m, k, mode="constant")
        ref_v = num_v / np.where(den > 0, den * den, 1)
        assert np.allclose(out[~bg, ch], ref_c[~bg], atol=1e-12)
        assert np.allclose(out[~bg, 2 + ch], ref_v[~bg], atol=1e-12)


def test_atrous_variance_closed_form(orc):
    """Constant variance v away from borders: v' = v (sum of squared taps)
    = v (1/16^2 * 2 + 1/4^2 * 2 + (3/8)^2)^2 = 0.07476806640625 v, and
    v (1/4^2 * 2 + 1/2^2)^2 = 0.140625 v for the 3x3 kernel."""
    H, W = 30, 30
    zn, _ = _flat_gbuffer(H, W)
    illum = np.full((H, W, 4), 0.5)
    illum[..., 2:] = 0.2
    out = orc.svgf_atrous(zn, illum, 1, orc.SvgfParams(**P_TEXTBOOK))
    assert np.allclose(out[5:-5, 5:-5, 2:], 0.2 * 0.07476806640625, atol=1e-15)
    out = orc.svgf_atrous(zn, illum, 1, orc.SvgfParams(kernel_width=3, **P_TEXTBOOK))
    assert np.allclose(out[5:-5, 5:-5, 2:], 0.2 * 0.140625, atol=1e-15)


def test_atrous_depth_edge_stops(orc):
    """Two fronto-parallel surfaces at depths 1 and 100: no weight crosses the
    depth discontinuity, so each side is filtered as if alone."""
    r = np.random.default_rng(11)
    H, W = 32, 40
    zn, _ = _flat_gbuffer(H, W)
    left = np.zeros((H, W), bool)
    left[:, :17] = True
    zn[left, 0] = 1.0
    zn[~left, 0] = 100.0
    illum = r.uniform(0.1, 1, (H, W, 4))
    for step in (1, 2, 4):
        out = orc.svgf_atrous(zn, illum, step, orc.SvgfParams(**P_TEXTBOOK))
        k = _dilated(step)
        for side in (left, ~left):
            ref = _normconv(illum[..., 0], side.astype(float), k)
            assert np.allclose(out[side, 0], ref[side], atol=1e-12)


def test_atrous_normal_edge_stops(orc):
    """Perpendicular normals give w_n = max(0, n.n')^sigma_n = 0 across the edge."""
    r = np.random.default_rng(12)
    H, W = 32, 40
    zn, _ = _flat_gbuffer(H, W)
    top = np.zeros((H, W), bool)
    top[:13] = True
    zn[top, 1:] = (1.0, 0.0, 0.0)
    illum = r.uniform(0.1, 1, (H, W, 4))
    out = orc.svgf_atrous(zn, illum, 2, orc.SvgfParams(sigma_n=128.0, sigma_l=1e30))
    k = _dilated(2)
    for side in (top, ~top):
        ref = _normconv(illum[..., 1], side.astype(float), k)
        assert np.allclose(out[side, 1], ref[side], atol=1e-12)


def test_atrous_luminance_stops_outlier(orc):
    """A bright outlier whose neighbourhood has near-zero variance receives
    almost no weight from its darker neighbours (w_l -> 0) and stays put,
    whereas without the luminance term it is blurred."""
    H, W = 21, 21
    zn, _ = _flat_gbuffer(H, W)
    illum = np.zeros((H, W, 4))
    illum[..., 0] = 0.2
    illum[10, 10, 0] = 0.9
    illum[..., 2] = 1e-8
    out = orc.svgf_atrous(zn, illum, 1, orc.SvgfParams(sigma_n=0.0, sigma_l=4.0))
    out2 = orc.svgf_atrous(zn, illum, 1, orc.SvgfParams(**P_TEXTBOOK))
    assert abs(out[10, 10, 0] - 0.9) < 1e-6
    assert abs(out2[10, 10, 0] - (0.2 + 0.7 * (3 / 8) ** 2)) < 1e-12


# --------------------------------------------------------------------------
# temporal accumulation and variance
# --------------------------------------------------------------------------
def _plane_view(orc, W=48, H=40, cam=None):
    """Oracle-traced G-buffer of a large quad facing +z seen by `cam`."""
    S = orc.Scene(wl.scene_quad([[-50, -50, -8], [50, -50, -8], [50, 50, -8], [-50, 50, -8]], 3))
    cam = cam or wl.look_at((0, 0, 0), (0, 0, -1), W, H)
    tr = orc.trace(S, cam, orc.TraceParams())
    zn, mesh = orc.gbuffer_f32(tr, cam.width, cam.height)
    return zn, mesh, cam


def _counts(r, H, W, spp=255):
    return r.integers(0, spp + 1, (H, W)).astype(np.uint8)


def test_temporal_fixed_alpha_geometric(orc):
    """Static camera, fixed alpha: four frames of input a, then constant c.
    From then on mu1 - c = (1 - alpha)^j (a - c) after j frames of c (Section
    3.3: exponential moving average); with history length >= 4 the colour is
    the same moving average (for shorter history it is the spatial mean,
    which equals a here)."""
    zn, mesh, cam = _plane_view(orc)
    H, W = mesh.shape
    st = orc.SvgfState(W, H)
    p = orc.SvgfParams(ao_spp=255, levels=0, fixed_alpha=True, alpha=0.2)
    a, c = 51 / 255, 204 / 255
    mask = np.zeros((H, W), np.uint8)
    for k in range(4):
        res = st.frame(zn, mesh, cam, mask, np.full((H, W), 51, np.uint8), p)
        assert np.allclose(st.mom[..., 0], a, atol=1e-12)
        assert np.allclose(res["ao"], a, atol=1e-12)
    for j in range(1, 12):
        res = st.frame(zn, mesh, cam, mask, np.full((H, W), 204, np.uint8), p)
        expect = c + 0.8 ** j * (a - c)
        assert np.allclose(st.mom[..., 0], expect, atol=1e-12)
        assert np.allclose(st.mom[..., 2], c * c + 0.8 ** j * (a * a - c * c), atol=1e-12)
        assert np.allclose(res["ao"], expect, atol=1e-12)


def test_temporal_ramp_is_running_mean_and_variance(orc):
    """alpha_eff = max(alpha, 1/n): for n <= 5 the moments are running means
    of s and s^2, so at n = 4, 5 the variance is the biased sample variance
    of the inputs so far; afterwards the EMA with alpha takes over.  The
    binary32 back-projection of a static camera lands within ~1e-5 px of the
    pixel centre, so neighbouring history leaks in at that level (tolerance
    2e-5 instead of rounding level)."""
    r = np.random.default_rng(5)
    zn, mesh, cam = _plane_view(orc)
    H, W = mesh.shape
    st = orc.SvgfState(W, H)
    p = orc.SvgfParams(ao_spp=255, levels=0)
    hist = []
    mask = np.zeros((H, W), np.uint8)
    for k in range(1, 8):
        ao = _counts(r, H, W)
        hist.append(ao / 255.0)
        res = st.frame(zn, mesh, cam, mask, ao, p)
        S = np.stack(hist)
        assert (st.hist == k).all()
        if k <= 5:
            assert np.allclose(st.mom[..., 0], S.mean(0), atol=2e-5)
            assert np.allclose(st.mom[..., 2], (S * S).mean(0), atol=2e-5)
        if k in (4, 5):
            assert np.allclose(res["illum"][..., 2], S.var(0), atol=2e-5)
            # colour: moving average (alpha_eff = 1/n) of last frame's colour
            exp_c = (1 - 1 / k) * prev_colour + (1 / k) * hist[-1]
            assert np.allclose(res["illum"][..., 0], exp_c, atol=2e-5)
        prev_colour = res["illum"][..., 0].copy()
        if k == 6:
            prev = np.stack(hist[:5]).mean(0)
            assert np.allclose(st.mom[..., 0], 0.8 * prev + 0.2 * hist[-1], atol=2e-5)


def test_spatial_variance_without_history(orc):
    """No history (n = 1 < 4): variance and colour come from a 7x7 window of
    the current frame weighted by depth and normal only; on a flat surface all
    weights are 1, giving the plain windowed mean and biased variance."""
    r = np.random.default_rng(8)
    H, W = 33, 45
    bg = r.random((H, W)) < 0.07
    zn, mesh = _flat_gbuffer(H, W, background=bg)
    ao = _counts(r, H, W)
    mask = r.integers(0, 2, (H, W)).astype(np.uint8)
    cam = wl.look_at((0, 0, 0), (0, 0, -1), W, H)
    res = orc.svgf_temporal(zn, mesh, cam, mask, ao, orc.SvgfParams(ao_spp=255))
    m = (~bg).astype(float)
    ones = np.ones((7, 7))
    for ch, s in enumerate([ao / 255.0, (mask & 1).astype(float)]):
        m1 = _normconv(s, m, ones)
        m2 = _normconv(s * s, m, ones)
        assert np.allclose(res["illum"][~bg, ch], m1[~bg], atol=1e-12)
        assert np.allclose(res["illum"][~bg, 2 + ch], np.maximum(0, m2 - m1 * m1)[~bg], atol=1e-12)
    assert (res["illum"][bg, :2] == 1).all()


def _shifted_cam(W, H, k_px, depth=8.0):
    """Camera translated along its right axis so that a fronto-parallel
    plane at `depth` moves by exactly k_px pixels on screen."""
    cam0 = wl.look_at((0, 0, 0), (0, 0, -1), W, H)
    t = cam0.tan_half_fov_y
    dx = k_px * 2.0 * depth * t * (W / H) / W
    return cam0, wl.look_at((dx, 0, 0), (dx, 0, -1), W, H)


def test_reprojection_follows_camera_shift(orc):
    """Section 3.3: the pixel's world position is back-projected into the
    previous frame.  A sideways camera move of exactly 3 pixels maps the
    history of pixel x + 3 onto pixel x; pixels whose history falls off
    screen restart (n = 1)."""
    W, H = 48, 40
    cam0, cam1 = _shifted_cam(W, H, 3)
    zn0, mesh0, _ = _plane_view(orc, cam=cam0)
    zn1, mesh1, _ = _plane_view(orc, cam=cam1)
    r = np.random.default_rng(9)
    ao0, ao1 = _counts(r, H, W), _counts(r, H, W)
    mask = np.zeros((H, W), np.uint8)
    p = orc.SvgfParams(ao_spp=255, levels=0)
    st = orc.SvgfState(W, H)
    st.frame(zn0, mesh0, cam0, mask, ao0, p)
    mu_prev = st.mom[..., 0].copy()
    res = orc.svgf_temporal(zn1, mesh1, cam1, mask, ao1, p, prev=(zn0, mesh0, cam0),
                            col_hist=st.col, mom=mu_prev[..., None].repeat(4, -1), hist=st.hist)
    inside = np.zeros((H, W), bool)
    inside[:, :W - 3] = True
    exp = 0.5 * np.roll(mu_prev, -3, axis=1) + 0.5 * ao1 / 255.0
    assert (res["valid"][inside] == 1).all()
    assert (res["hist"][inside] == 2).all()
    assert np.allclose(res["mom"][inside, 0], exp[inside], atol=2e-5)
    assert (res["hist"][:, W - 2:] == 1).all()
    assert np.allclose(res["mom"][:, W - 2:, 0], (ao1 / 255.0)[:, W - 2:], atol=1e-12)


@pytest.mark.parametrize("change,valid", [("mesh", False), ("depth+2%", False), ("depth+0.5%", True),
                                          ("normal30", False), ("normal20", True)])
def test_reprojection_rejects_inconsistent_history(orc, change, valid):
    """History taps are discarded when mesh id, projected depth (1 %) or
    normal (cos < 0.9) disagree (Section 3.3)."""
    zn, mesh, cam = _plane_view(orc)
    H, W = mesh.shape
    znp, meshp = zn.copy(), mesh.copy()
    if change == "mesh":
        meshp = meshp + 1
    elif change.startswith("depth"):
        znp[..., 0] *= 1.02 if "2%" in change else 1.005
    else:
        a = math.radians(30 if "30" in change else 20)
        znp[..., 1:] = (math.sin(a), 0.0, math.cos(a))
    ao = np.full((H, W), 100, np.uint8)
    res = orc.svgf_temporal(zn, mesh, cam, np.zeros((H, W), np.uint8), ao,
                            orc.SvgfParams(ao_spp=255), prev=(znp, meshp, cam),
                            hist=np.full((H, W), 7, np.int32))
    assert (res["valid"] == int(valid)).all()
    assert (res["hist"] == (8 if valid else 1)).all()


def test_svgf_output_is_convex(orc):
    """Every stage is a normalised non-negative combination of inputs in
    [0, 1], so the filtered AO and shadow stay in [0, 1]."""
    s = wl.scene_boxes()
    S = orc.Scene(s)
    cams = wl.orbit_path(3, 64, 64)
    st = orc.SvgfState(64, 64)
    for f, cam in enumerate(cams):
        tr = orc.trace(S, cam, orc.TraceParams(frame=f))
        zn, mesh = orc.gbuffer_f32(tr, 64, 64)
        res = st.frame(zn, mesh, cam, tr["shadow_mask"].reshape(64, 64),
                       tr["ao_count"].reshape(64, 64), orc.SvgfParams())
        for k in ("ao", "shadow"):
            assert res[k].min() >= -1e-12 and res[k].max() <= 1 + 1e-12


@pytest.mark.parametrize("step", [1, 2, 4])
@pytest.mark.parametrize("sigma_z", [1.0, 2.5])
def test_atrous_depth_weight_on_a_tilted_plane(orc, step, sigma_z):
    """Depth linear in the pixel coordinates, z = 10 + x/4 + y/32 (exact in
    binary32): the one-sided differences are the gradient, |z_p - z_q| =
    |grad z . (p - q)| at every tap, so with eps_z = 0 the depth weight is
    w_z = exp(-1 / sigma_z) for every tap but the centre (Section 3.3).  With
    w_n = w_l = 1 the pass is the B3 kernel with its off-centre taps scaled
    by that constant; colour and variance follow in closed form."""
    r = np.random.default_rng(20 + step)
    H, W = 36, 44
    ys, xs = np.mgrid[0:H, 0:W]
    zn, _ = _flat_gbuffer(H, W)
    zn[..., 0] = (10.0 + xs / 4.0 + ys / 32.0).astype(np.float32)
    illum = r.uniform(0.05, 1, (H, W, 4))
    out = orc.svgf_atrous(zn, illum, step, orc.SvgfParams(sigma_z=sigma_z, eps_z=0.0, **P_TEXTBOOK))
    E = math.exp(-1.0 / sigma_z)
    k = _dilated(step)
    kc = (3 / 8) ** 2
    wk = k * E
    wk[2 * step, 2 * step] = kc           # the centre tap keeps its kernel weight
    m = 2 * step
    inner = (slice(m, H - m), slice(m, W - m))
    for ch in range(2):
        num = ndimage.correlate(illum[..., ch], wk, mode="constant")
        num_v = ndimage.correlate(illum[..., 2 + ch], wk * wk, mode="constant")
        den = kc + E * (1 - kc)
        assert np.allclose(out[inner + (ch,)], (num / den)[inner], atol=1e-12)
        assert np.allclose(out[inner + (2 + ch,)], (num_v / den ** 2)[inner], atol=1e-12)


@pytest.mark.parametrize("step", [1, 2])
def test_atrous_ridge_is_filtered_along_itself(orc, step):
    """A one-pixel column one unit in front of a fronto-parallel plane (depth
    10 -> 9).  On the column the horizontal one-sided depth differences are
    +1 and -1, so its depth slope is 0 (minmod) and every tap off the column
    has w_z = exp(-1 / eps_z) = exp(-100): the column is filtered along
    itself only, by the 1-D B3 kernel.  Beside it one difference is 0, so the
    slope is 0 there too and the plane never takes the column's taps."""
    r = np.random.default_rng(30 + step)
    H, W = 40, 48
    zn, _ = _flat_gbuffer(H, W, depth=10.0)
    c = 23
    zn[:, c, 0] = 9.0
    illum = r.uniform(0.05, 1, (H, W, 4))
    out = orc.svgf_atrous(zn, illum, step, orc.SvgfParams(**P_TEXTBOOK))
    k1 = np.zeros(4 * step + 1)
    k1[::step] = B3
    col = np.zeros((H, W))
    col[:, c] = 1.0
    k2 = np.zeros((len(k1), len(k1)))
    k2[:, 2 * step] = k1                   # vertical taps only
    for ch in range(2):
        ref_col = _normconv(illum[..., ch], col, k2)
        assert np.allclose(out[:, c, ch], ref_col[:, c], atol=1e-12)
        plane = 1.0 - col
        ref_plane = _normconv(illum[..., ch], plane, _dilated(step))
        m = plane.astype(bool)
        assert np.allclose(out[m, ch], ref_plane[m], atol=1e-12)
