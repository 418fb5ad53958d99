"""Pins for the oracle's hand-derived adjoint of the modified SVGF.

The adjoint (dL/ds for every noisy input and dL/d sigma_z, sigma_n,
sigma_l, through the temporal recursion and all a-trous levels) is checked
against central finite differences of the oracle's own double-precision
forward, and against the linearity of the loss in g_out.
"""
import numpy as np
import pytest

import oracle as orc
import workloads as wl


def _scene():
    """Boxes plus three level-2 icospheres (curved surfaces: n.n' < 1 between
    neighbouring pixels, so the sigma_n gradient is exercised)."""
    b = wl.scene_boxes()
    v, t = wl.icosphere(2)
    parts = [b]
    for k, (c, r) in enumerate((((0.0, 1.0, 0.0), 1.0), ((1.8, 0.6, 1.2), 0.6), ((-1.5, 0.8, 0.8), 0.8))):
        parts.append(dict(vertices=(v * r + np.array(c)).astype(np.float32), indices=t.astype(np.uint32),
                          mesh_ids=np.full(len(t), 100 + k, np.uint32)))
    return wl.merge(*parts)


def _sequence(W=28, H=20, F=6, seed=0):
    S = orc.Scene(_scene())
    cams = wl.orbit_path(F, W, H, degrees=3.0, radius=5.0, height_y=2.5)
    zn, mesh = [], []
    for f, cam in enumerate(cams):
        tr = orc.trace(S, cam, orc.TraceParams(frame=f))
        z, m = orc.gbuffer_f32(tr, W, H)
        zn.append(z)
        mesh.append(m)
    r = np.random.default_rng(seed)
    sig = r.uniform(0.05, 0.95, (F, H, W, 2))
    g_out = r.normal(size=(F, H, W, 2))
    return np.stack(zn), np.stack(mesh), cams, sig, g_out


def _loss(zn, mesh, cams, sig, params, g_out):
    out, _, _ = orc.svgf_seq_grad(zn, mesh, cams, sig, params, np.zeros_like(g_out))
    return float((out * g_out).sum())


@pytest.mark.parametrize("levels,wl_in", [(3, True), (5, True), (2, False)])
def test_adjoint_matches_finite_differences(levels, wl_in):
    zn, mesh, cams, sig, g_out = _sequence()
    p = orc.SvgfParams(levels=levels, wl_in_atrous=wl_in)
    out, g_sig, g_sigma = orc.svgf_seq_grad(zn, mesh, cams, sig, p, g_out)
    fg = np.isfinite(zn[..., 0])
    assert fg.mean() > 0.5
    # both variance paths run: short history (frames 0-2) and moments (n >= 4)
    st = orc.SvgfState(zn.shape[2], zn.shape[1])
    for f in range(len(cams)):
        st.frame(zn[f], mesh[f], cams[f], np.zeros(zn.shape[1:3], np.uint8),
                 np.zeros(zn.shape[1:3], np.uint8), p)
    assert (st.hist >= 4).sum() > 100
    assert abs(g_sigma[0]) > 1e-3 and abs(g_sigma[1]) > 1e-6
    r = np.random.default_rng(1)
    idx = np.argwhere(np.broadcast_to(fg[..., None], sig.shape))
    pick = idx[r.choice(len(idx), 30, replace=False)]
    h = 1e-6
    for f, y, x, c in pick:
        sp, sm = sig.copy(), sig.copy()
        sp[f, y, x, c] += h
        sm[f, y, x, c] -= h
        fd = (_loss(zn, mesh, cams, sp, p, g_out) - _loss(zn, mesh, cams, sm, p, g_out)) / (2 * h)
        an = g_sig[f, y, x, c]
        assert abs(fd - an) <= 1e-5 * (1.0 + abs(an)), (f, y, x, c, fd, an)
    for k, name in enumerate(("sigma_z", "sigma_n", "sigma_l")):
        if name == "sigma_l" and not wl_in:
            assert g_sigma[2] == 0.0
            continue
        base = getattr(p, name)
        hh = 1e-6 * base
        pp = orc.SvgfParams(**{**p.__dict__, name: base + hh})
        pm = orc.SvgfParams(**{**p.__dict__, name: base - hh})
        fd = (_loss(zn, mesh, cams, sig, pp, g_out) - _loss(zn, mesh, cams, sig, pm, g_out)) / (2 * hh)
        assert abs(fd - g_sigma[k]) <= 1e-4 * (1.0 + abs(g_sigma[k])), (name, fd, g_sigma[k])


def test_adjoint_forward_equals_frame_by_frame_oracle():
    """The sequence forward inside the adjoint is the same filter as the
    per-frame oracle (fed the same signals as 8-bit counts)."""
    zn, mesh, cams, _, g_out = _sequence()
    F, H, W = zn.shape[:3]
    r = np.random.default_rng(3)
    cnt = r.integers(0, 256, (F, H, W)).astype(np.uint8)
    mask = r.integers(0, 2, (F, H, W)).astype(np.uint8)
    sig = np.stack([cnt / 255.0, (mask & 1).astype(float)], -1)
    p = orc.SvgfParams(ao_spp=255)
    out, _, _ = orc.svgf_seq_grad(zn, mesh, cams, sig, p, g_out)
    st = orc.SvgfState(W, H)
    for f in range(F):
        ref = st.frame(zn[f], mesh[f], cams[f], mask[f], cnt[f], p)
        assert np.allclose(out[f, ..., 0], ref["ao"], atol=1e-12)
        assert np.allclose(out[f, ..., 1], ref["shadow"], atol=1e-12)


def test_adjoint_is_linear_in_upstream_gradient():
    zn, mesh, cams, sig, g1 = _sequence(seed=4)
    g2 = np.random.default_rng(9).normal(size=g1.shape)
    p = orc.SvgfParams(levels=3)
    _, a1, s1 = orc.svgf_seq_grad(zn, mesh, cams, sig, p, g1)
    _, a2, s2 = orc.svgf_seq_grad(zn, mesh, cams, sig, p, g2)
    _, a3, s3 = orc.svgf_seq_grad(zn, mesh, cams, sig, p, 2.0 * g1 - 0.5 * g2)
    assert np.allclose(a3, 2.0 * a1 - 0.5 * a2, atol=1e-10)
    assert np.allclose(s3, 2.0 * s1 - 0.5 * s2, rtol=1e-9, atol=1e-10)
