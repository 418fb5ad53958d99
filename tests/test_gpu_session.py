"""dhr_step_frame (trace + SVGF with library-owned ping-pong buffers) gives
exactly what the two component calls give, and the host-output variant
returns the same bytes."""
import numpy as np
import pytest

import paper_2406_06963_b300 as dhrs
import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_step_frame_equals_components():
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    W, H = 160, 96
    cams = wl.orbit_path(5, W, H, degrees=6.0)
    tp = dhrs.TraceParams(ao_spp=2)
    sp = dhrs.SvgfParams(ao_spp=2)
    sess = dhrs.Session(sc, W, H, dhrs.DHR_FP32, tp, sp)
    st = dhrs.SvgfState(W, H)
    a1, s1 = torch.empty((H, W), device="cuda"), torch.empty((H, W), device="cuda")
    a2, s2 = torch.empty_like(a1), torch.empty_like(a1)
    prev = None
    for f, cam in enumerate(cams):
        sess.step(cam, f, a1, s1)
        g = dhrs.GBuffer(W, H)
        m = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        a = torch.empty_like(m)
        tpf = dhrs.TraceParams(ao_spp=2, frame=f)
        dhrs.trace_visibility(sc, cam, tpf, g, m, a)
        st.reconstruct(g, prev[0] if prev else None, cam, prev[1] if prev else None, m, a, sp, a2, s2)
        prev = (g, cam)
        torch.cuda.synchronize()
        assert torch.equal(a1, a2) and torch.equal(s1, s2), f
    ah = torch.empty((H, W), pin_memory=True)
    sh = torch.empty((H, W), pin_memory=True)
    sess2 = dhrs.Session(sc, W, H, dhrs.DHR_FP32, tp, sp)
    for f, cam in enumerate(cams):
        sess2.step_host(cam, f, ah, sh)
    assert torch.equal(ah, a1.cpu()) and torch.equal(sh, s1.cpu())


def test_session_reset_drops_history():
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    cam = wl.boxes_camera(64, 64)
    sess = dhrs.Session(sc, 64, 64)
    o1 = torch.empty((64, 64), device="cuda")
    o2 = torch.empty_like(o1)
    sh = torch.empty_like(o1)
    sess.step(cam, 0, o1, sh)
    sess.step(cam, 1, o2, sh)
    sess.reset()
    o3 = torch.empty_like(o1)
    sess.step(cam, 0, o3, sh)          # same frame index, no history: same as the first frame
    torch.cuda.synchronize()
    assert torch.equal(o1, o3)
    assert not torch.equal(o1, o2)


def test_streaming_host_output_equals_synchronous():
    """dhr_step_frame_host_async with two alternating pinned buffers returns,
    after dhr_session_wait, exactly what the synchronous host path returns;
    tickets increase and an unissued ticket is rejected."""
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    W, H = 160, 96
    cams = wl.orbit_path(6, W, H, degrees=6.0)
    ref = dhrs.Session(sc, W, H)
    a_ref = [torch.empty((H, W), pin_memory=True) for _ in cams]
    s_ref = [torch.empty((H, W), pin_memory=True) for _ in cams]
    for f, cam in enumerate(cams):
        ref.step_host(cam, f, a_ref[f], s_ref[f])
    sess = dhrs.Session(sc, W, H)
    bufs = [(torch.empty((H, W), pin_memory=True), torch.empty((H, W), pin_memory=True)) for _ in range(2)]
    prev = None
    for f, cam in enumerate(cams):
        ab, sb = bufs[f & 1]
        t = sess.step_host_async(cam, f, ab, sb)
        assert t == f + 1
        if prev is not None:
            pf, pt = prev
            sess.wait(pt)
            pa, ps = bufs[pf & 1]
            assert torch.equal(pa, a_ref[pf]) and torch.equal(ps, s_ref[pf]), pf
        prev = (f, t)
    sess.wait(prev[1])
    pa, ps = bufs[prev[0] & 1]
    assert torch.equal(pa, a_ref[prev[0]]) and torch.equal(ps, s_ref[prev[0]])
    with pytest.raises(dhrs.DhrError):
        sess.wait(prev[1] + 1)
    # the synchronous path on the same session still works after streaming
    a2, s2 = torch.empty((H, W), pin_memory=True), torch.empty((H, W), pin_memory=True)
    sess.step_host(cams[0], 99, a2, s2)
    assert bool(torch.isfinite(a2).all())


def test_step_frame_sequence_matches_oracle():
    """Six pipelined, rasterised dhr_step_frame frames of the box scene
    against the oracle tracing the same frames itself and filtering them
    with orc_svgf_frame (Sections 3.1-3.3 end to end).  The raw trace
    outputs must equal the oracle's except on rays it flags as grazing; the
    filtered AO and shadow must be within 1e-3 of the oracle's on every
    pixel whose filter footprint, over all frames so far, saw no such ray
    (a flipped bit spreads through the a-trous levels up to 62 pixels away
    and through the history)."""
    import oracle as orc
    s = wl.scene_boxes()
    sc, S = dhrs.Scene(s), orc.Scene(s)
    W, H = 256, 192
    cams = wl.orbit_path(6, W, H, degrees=10.0)
    sess = dhrs.Session(sc, W, H)
    ost = orc.SvgfState(W, H)
    ao, sh = torch.empty((H, W), device="cuda"), torch.empty((H, W), device="cuda")
    tainted = np.zeros((H, W), bool)
    checked = 0
    for f, cam in enumerate(cams):
        sess.step(cam, f, ao, sh)
        tr = orc.trace(S, cam, orc.TraceParams(frame=f))
        zn, mesh = orc.gbuffer_f32(tr, W, H)
        mask, cnt = tr["shadow_mask"].reshape(H, W), tr["ao_count"].reshape(H, W)
        ref = ost.frame(zn, mesh, cam, mask, cnt, orc.SvgfParams())
        torch.cuda.synchronize()
        fb = sess.frame_buffers()
        g_mask = dhrs.device_copy(fb["mask"], (H, W), "uint8").cpu().numpy()
        g_ao = dhrs.device_copy(fb["ao"], (H, W), "uint8").cpu().numpy()
        flagged = (tr["amb_primary"] | tr["amb_shadow"] | tr["amb_ao"]).reshape(H, W) > 0
        differ = (g_mask != mask) | (g_ao != cnt)
        assert not (differ & ~flagged).any(), f
        if differ.any():
            ys, xs = np.nonzero(differ)
            for y, x in zip(ys, xs):
                tainted[max(0, y - 72):y + 73, max(0, x - 72):x + 73] = True
        ok = ~tainted
        e = np.maximum(np.abs(ao.cpu().numpy() - ref["ao"]), np.abs(sh.cpu().numpy() - ref["shadow"]))
        assert e[ok].max() <= 1e-3, (f, float(e[ok].max()))
        checked += int(ok.sum())
    assert checked >= 0.9 * W * H * len(cams)


@pytest.mark.parametrize("precision", [dhrs.DHR_FP32, dhrs.DHR_FP16])
def test_checkpoint_resume_continues_exactly(precision):
    """A session exported after three frames and imported into a fresh
    session continues bit for bit as the original does (same cameras and
    parameters); a checkpoint of another size or a damaged one is refused."""
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    W, H = 160, 96
    cams = wl.orbit_path(6, W, H, degrees=8.0)
    a = dhrs.Session(sc, W, H, precision)
    o = [torch.empty((H, W), device="cuda") for _ in range(4)]
    for f in range(3):
        a.step(cams[f], f, o[0], o[1])
    image = a.checkpoint()
    assert image.size == dhrs.lib().dhr_session_checkpoint_bytes(a.h)
    b = dhrs.Session(sc, W, H, precision)
    b.restore(image)
    for f in range(3, 6):
        a.step(cams[f], f, o[0], o[1])
        b.step(cams[f], f, o[2], o[3])
        torch.cuda.synchronize()
        assert torch.equal(o[0], o[2]) and torch.equal(o[1], o[3]), f
    # a fresh session without the checkpoint differs (the history matters)
    c = dhrs.Session(sc, W, H, precision)
    c.step(cams[5], 5, o[2], o[3])
    torch.cuda.synchronize()
    assert not torch.equal(o[0], o[2])
    other = dhrs.Session(sc, W + 8, H, precision)
    with pytest.raises(dhrs.DhrError):
        other.restore(image)
    bad = image.copy()
    bad[0] ^= 0xFF
    with pytest.raises(dhrs.DhrError):
        b.restore(bad)
    with pytest.raises(dhrs.DhrError):
        b.restore(image[:100])
