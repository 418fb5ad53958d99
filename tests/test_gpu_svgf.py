"""GPU parity of the modified SVGF (Section 3.3) against the CPU oracle.

Both sides get the same inputs: a G-buffer and noisy AO/shadow traced by
the oracle, rounded to binary32 (the CUDA path's storage).  Bar: filtered AO
and shadow within 1e-3 absolute of the fp64 oracle on every pixel of every
frame; history length and validity identical (binary32 reprojection
decisions are specified identically on both sides).
"""
import numpy as np
import pytest

import oracle as orc
import paper_2406_06963_b300 as dhrs
import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-3


def _oracle_frames(scene, cams, tp_kw=None):
    S = orc.Scene(scene)
    out = []
    for f, cam in enumerate(cams):
        tr = orc.trace(S, cam, orc.TraceParams(frame=f, **(tp_kw or {})))
        zn, mesh = orc.gbuffer_f32(tr, cam.width, cam.height)
        out.append((zn, mesh, tr["shadow_mask"].reshape(cam.height, cam.width),
                    tr["ao_count"].reshape(cam.height, cam.width)))
    return out


def _run_both(frames, cams, op: "orc.SvgfParams", precision=dhrs.DHR_FP32, check_internal=True, shadow_light=0):
    """shadow_light = k: the GPU filters bit k of the full bitmask, the oracle
    (which filters bit 0) is given the bitmask shifted right by k."""
    W, H = cams[0].width, cams[0].height
    ost = orc.SvgfState(W, H)
    gst = dhrs.SvgfState(W, H, precision)
    gp = dhrs.SvgfParams(**op.__dict__, shadow_light=shadow_light)
    prev = None
    worst = 0.0
    ao_o = torch.empty((H, W), device="cuda")
    sh_o = torch.empty((H, W), device="cuda")
    for f, (zn, mesh, mask, ao) in enumerate(frames):
        ref = ost.frame(zn, mesh, cams[f], mask >> shadow_light, ao, op)
        g = dhrs.GBuffer.from_arrays(zn, mesh, precision)
        gst.reconstruct(g, prev[0] if prev else None, cams[f], prev[1] if prev else None,
                        torch.from_numpy(mask).cuda(), torch.from_numpy(ao).cuda(), gp, ao_o, sh_o)
        torch.cuda.synchronize()
        fg = np.isfinite(zn[..., 0])
        e_ao = np.abs(ao_o.cpu().numpy() - ref["ao"])
        e_sh = np.abs(sh_o.cpu().numpy() - ref["shadow"])
        worst = max(worst, float(e_ao.max()), float(e_sh.max()))
        if check_internal and precision == dhrs.DHR_FP32:
            b = gst.buffers()
            hist = dhrs.device_copy(b["histlen"], (H, W), "uint8").cpu().numpy()
            assert np.array_equal(hist.astype(np.int32), np.where(fg, ost.hist, 0)), f
            illum = dhrs.device_copy(b["illum"], (H, W, 4), "float32").cpu().numpy()
            # the temporal colour carries last frame's level-0 colour, so it
            # inherits that pass's binary32 accumulation error
            assert np.abs(illum - ref["illum"])[fg].max() < 5e-4, f
        prev = (g, cams[f])
    print(f"svgf parity {W}x{H} x{len(frames)} frames: max |gpu - oracle| = {worst:.3g}")
    return worst


def test_svgf_boxes_sequence():
    """256x256, 194 triangles, 8 frames of a slow orbit (history valid,
    disocclusions at box edges), 5 a-trous levels."""
    s = wl.scene_boxes()
    cams = wl.orbit_path(8, 256, 256, degrees=8.0)
    frames = _oracle_frames(s, cams)
    assert _run_both(frames, cams, orc.SvgfParams()) <= TOL


@pytest.mark.parametrize("levels", [0, 1, 2, 5])
def test_svgf_ragged_and_levels(levels):
    s = wl.scene_boxes()
    cams = wl.orbit_path(5, 37, 23, degrees=10.0)
    frames = _oracle_frames(s, cams)
    assert _run_both(frames, cams, orc.SvgfParams(levels=levels)) <= TOL


@pytest.mark.parametrize("levels,size", [(1, (96, 64)), (5, (96, 64)), (1, (37, 23)), (2, (37, 23))])
def test_svgf_small_kernel(levels, size):
    """The lightweight denoiser's smaller kernel (3x3 taps 1/4, 1/2, 1/4;
    Section 3.3), one level as proposed and more, full and ragged images."""
    s = wl.scene_boxes()
    cams = wl.orbit_path(5, *size, degrees=8.0)
    frames = _oracle_frames(s, cams)
    assert _run_both(frames, cams, orc.SvgfParams(levels=levels, kernel_width=3)) <= TOL


def test_svgf_fixed_alpha_no_luminance_multi_spp():
    s = wl.scene_boxes()
    cams = wl.orbit_path(6, 96, 64, degrees=6.0)
    frames = _oracle_frames(s, cams, dict(ao_spp=8))
    p = orc.SvgfParams(ao_spp=8, fixed_alpha=True, wl_in_atrous=False, sigma_n=32.0, sigma_z=2.0)
    assert _run_both(frames, cams, p) <= TOL


@pytest.mark.parametrize("light", [1, 2])
def test_svgf_filters_the_selected_light(light):
    """Three lights with different cone angles: shadow_light = k filters bit k
    of the visibility bitmask (the oracle gets that bit as its bit 0)."""
    s = wl.scene_boxes()
    cams = wl.orbit_path(4, 96, 64, degrees=6.0)
    tp = dict(light_dirs=[(0.3, 1.0, 0.2), (-0.6, 0.8, 0.3), (0.2, 0.5, -0.8)],
              cone_half_angle_deg=[0.5, 3.0, 1.5])
    frames = _oracle_frames(s, cams, tp)
    bits = np.stack([f[2] for f in frames])
    assert ((bits >> light) & 1).mean() != (bits & 1).mean()      # the lights differ
    assert _run_both(frames, cams, orc.SvgfParams(), shadow_light=light) <= TOL


@pytest.mark.slow
def test_svgf_1080p():
    """Full 1920x1080 frames (the launch configuration bench.py times), 3
    frames, against the full-frame oracle."""
    s = wl.scene_boxes()
    cams = wl.orbit_path(3, 1920, 1080, degrees=2.0)
    frames = _oracle_frames(s, cams)
    assert _run_both(frames, cams, orc.SvgfParams(), check_internal=False) <= TOL


def test_svgf_rejects_bad_arguments():
    st = dhrs.SvgfState(16, 16)
    g = dhrs.GBuffer(16, 16)
    cam = wl.boxes_camera(16, 16)
    m = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    o = torch.empty((16, 16), device="cuda")
    for bad in (dict(levels=9), dict(ao_spp=0), dict(alpha=0.0), dict(shadow_light=8), dict(kernel_width=4),
                dict(eps_z=0.0), dict(eps_l=0.0), dict(eps_z=float("inf"))):
        with pytest.raises(dhrs.DhrError):
            st.reconstruct(g, None, cam, None, m, m, dhrs.SvgfParams(**bad), o, o)
    g16 = dhrs.GBuffer(16, 16, dhrs.DHR_FP16)
    with pytest.raises(dhrs.DhrError):
        st.reconstruct(g16, None, cam, None, m, m, dhrs.SvgfParams(), o, o)


@pytest.mark.slow
def test_svgf_terrain_spline_1080p():
    """Three consecutive frames of the terrain camera spline at 1920x1080, the
    launch configuration bench.py times, on a coarse version of the terrain
    scene the brute-force oracle can trace in seconds: the same seeded
    heightfield on a 24 x 24 vertex grid with 8 icospheres and 8 boxes
    (1,794 triangles).  Distant terrain seen 25 degrees down exercises the
    depth-slope term of the reprojection test; history lengths must be
    identical and the filtered outputs within 1e-3 everywhere."""
    s = wl.scene_terrain(n_spheres=8, n_boxes=8, sphere_level=1, terrain_n=24)
    cams = wl.spline_path(s["terrain"], 60, 1920, 1080)[:3]
    frames = _oracle_frames(s, cams)
    assert _run_both(frames, cams, orc.SvgfParams()) <= TOL
