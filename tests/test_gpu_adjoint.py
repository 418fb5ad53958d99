"""GPU adjoint of the modified SVGF against the oracle's fp64 adjoint (which
is itself pinned by finite differences), and the torch.autograd path.

Same inputs on both sides: G-buffers traced by the oracle (binary32),
real-valued noisy signals, a random upstream gradient.  Bars: filtered
output within 1e-3; dL/d signal within 1e-3 of the largest oracle entry;
dL/d sigma within 1e-2 relative (binary32 sums over every pixel, level and
frame).
"""
import numpy as np
import pytest

import oracle as orc
import paper_2406_06963_b300 as dhrs
import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _scene():
    b = wl.scene_boxes()
    v, t = wl.icosphere(2)
    parts = [b]
    for k, (c, r) in enumerate((((0.0, 1.0, 0.0), 1.0), ((1.8, 0.6, 1.2), 0.6), ((-1.5, 0.8, 0.8), 0.8))):
        parts.append(dict(vertices=(v * r + np.array(c)).astype(np.float32), indices=t.astype(np.uint32),
                          mesh_ids=np.full(len(t), 100 + k, np.uint32)))
    return wl.merge(*parts)


def _inputs(W, H, F, seed=0):
    S = orc.Scene(_scene())
    cams = wl.orbit_path(F, W, H, degrees=4.0, radius=5.0, height_y=2.5)
    zn, mesh = [], []
    for f, cam in enumerate(cams):
        tr = orc.trace(S, cam, orc.TraceParams(frame=f))
        z, m = orc.gbuffer_f32(tr, W, H)
        zn.append(z)
        mesh.append(m)
    r = np.random.default_rng(seed)
    sig = r.uniform(0.02, 0.98, (F, H, W, 2))
    g_out = r.normal(size=(F, H, W, 2))
    return np.stack(zn), np.stack(mesh), cams, sig, g_out


def _planes(a):          # [F, H, W, 2] -> [F, 2, H, W]
    return np.ascontiguousarray(np.moveaxis(a, -1, 1))


@pytest.mark.parametrize("levels,wl_in,sigma_n,schedule", [
    (5, True, 128.0, dhrs.TAPE_RECOMPUTE), (5, True, 128.0, dhrs.TAPE_STORE),
    (2, True, 128.0, dhrs.TAPE_RECOMPUTE), (3, False, 128.0, dhrs.TAPE_STORE),
    (1, True, 128.0, dhrs.TAPE_RECOMPUTE), (1, False, 128.0, dhrs.TAPE_STORE),
    (0, True, 128.0, dhrs.TAPE_RECOMPUTE), (3, True, 32.0, dhrs.TAPE_RECOMPUTE),
    (2, False, 0.0, dhrs.TAPE_STORE)])
def test_adjoint_matches_oracle(levels, wl_in, sigma_n, schedule):
    """sigma_n 128 takes the kernels' power-of-two normal weight; 32 and 0
    (no normal term) the general one.  Both record schedules: levels
    recomputed by the backward, and stored by the forward."""
    W, H, F = 64, 40, 6
    zn, mesh, cams, sig, g_out = _inputs(W, H, F)
    op = orc.SvgfParams(levels=levels, wl_in_atrous=wl_in, sigma_n=sigma_n)
    out_o, gsig_o, gsigma_o = orc.svgf_seq_grad(zn, mesh, cams, sig, op, g_out)
    gbufs = [dhrs.GBuffer.from_arrays(zn[f], mesh[f]) for f in range(F)]
    gp = dhrs.SvgfParams(**op.__dict__)
    tape = dhrs.SvgfTape(W, H, F, schedule)
    sig_t = torch.from_numpy(_planes(sig).astype(np.float32)).cuda()
    gout_t = torch.from_numpy(_planes(g_out).astype(np.float32)).cuda()
    out = tape.forward(gbufs, cams, sig_t, gp)
    g_sig, g_sigma = tape.backward(gbufs, cams, sig_t, gp, gout_t)
    torch.cuda.synchronize()
    out = np.moveaxis(out.cpu().numpy(), 1, -1)
    g_sig = np.moveaxis(g_sig.cpu().numpy(), 1, -1)
    g_sigma = g_sigma.cpu().numpy()
    e_out = np.abs(out - out_o).max()
    e_sig = np.abs(g_sig - gsig_o).max() / np.abs(gsig_o).max()
    print(f"adjoint L={levels} wl={wl_in}: out {e_out:.3g}, dL/ds rel {e_sig:.3g}, "
          f"dL/dsigma gpu {g_sigma} oracle {gsigma_o}")
    assert e_out <= 1e-3
    assert e_sig <= 1e-3
    for k in range(3):
        if gsigma_o[k] == 0.0:
            assert abs(g_sigma[k]) < 1e-6
        else:
            assert abs(g_sigma[k] - gsigma_o[k]) <= 1e-2 * abs(gsigma_o[k]) + 1e-4, (k, g_sigma, gsigma_o)


def test_autograd_function_and_fit():
    """torch.autograd path gives the tape's gradients, and a few Adam steps on
    log(sigma) lower the L2 loss against a many-sample reference."""
    W, H, F = 64, 40, 5
    zn, mesh, cams, sig, _ = _inputs(W, H, F, seed=2)
    gbufs = [dhrs.GBuffer.from_arrays(zn[f], mesh[f]) for f in range(F)]
    ref = torch.from_numpy(_planes(np.full_like(sig, 0.5)).astype(np.float32)).cuda()
    sig_t = torch.from_numpy(_planes(sig).astype(np.float32)).cuda().requires_grad_(True)
    log_s = torch.tensor(np.log([1.0, 128.0, 4.0]), dtype=torch.float32, device="cuda", requires_grad=True)
    tape = dhrs.SvgfTape(W, H, F)
    out = dhrs.svgf_sequence(sig_t, log_s.exp(), gbufs, cams, dhrs.SvgfParams(), tape)
    loss = ((out - ref) ** 2).sum()
    loss.backward()
    g_sig, g_sigma = tape.backward(gbufs, cams, sig_t.detach(), dhrs.SvgfParams(), 2 * (out - ref).detach())
    assert torch.allclose(sig_t.grad, g_sig, atol=1e-6)
    assert torch.allclose(log_s.grad, g_sigma * log_s.detach().exp(), rtol=1e-5, atol=1e-6)
    opt = torch.optim.Adam([log_s], lr=0.1)
    losses = []
    for _ in range(8):
        opt.zero_grad()
        out = dhrs.svgf_sequence(sig_t.detach(), log_s.exp(), gbufs, cams, dhrs.SvgfParams(), tape)
        l = ((out - ref) ** 2).sum()
        l.backward()
        opt.step()
        losses.append(float(l.detach()))
    print("fit losses", losses)
    assert losses[-1] < losses[0]


def test_recompute_schedule_equals_store():
    """The recomputed level records are the stored ones: the same filtered
    output bit for bit, the same gradients up to the atomics' summation
    order; a second backward after one forward gives the first's; the
    recomputing tape keeps two frames of level records, the storing one F."""
    W, H, F, L = 96, 56, 5, 5
    zn, mesh, cams, sig, g_out = _inputs(W, H, F, seed=4)
    gbufs = [dhrs.GBuffer.from_arrays(zn[f], mesh[f]) for f in range(F)]
    gp = dhrs.SvgfParams(levels=L, sigma_n=32.0)
    sig_t = torch.from_numpy(_planes(sig).astype(np.float32)).cuda()
    gout_t = torch.from_numpy(_planes(g_out).astype(np.float32)).cuda()
    res = {}
    for sched in (dhrs.TAPE_RECOMPUTE, dhrs.TAPE_STORE):
        tape = dhrs.SvgfTape(W, H, F, sched)
        out = tape.forward(gbufs, cams, sig_t, gp)
        g1 = tape.backward(gbufs, cams, sig_t, gp, gout_t)
        g2 = tape.backward(gbufs, cams, sig_t, gp, gout_t)
        torch.cuda.synchronize()
        res[sched] = (out, g1, g2, tape.level_bytes(L))
    N = W * H
    per_frame = N * (16 * (L - 1) + 8 * L + 16)
    assert res[dhrs.TAPE_RECOMPUTE][3] == 2 * per_frame
    assert res[dhrs.TAPE_STORE][3] == F * per_frame
    out_r, out_s = res[dhrs.TAPE_RECOMPUTE][0], res[dhrs.TAPE_STORE][0]
    assert torch.equal(out_r, out_s)
    ref_sig, ref_sigma = res[dhrs.TAPE_STORE][1]
    scale = float(ref_sig.abs().max())
    for sched in res:
        for g_sig, g_sigma in res[sched][1:3]:
            assert float((g_sig - ref_sig).abs().max()) <= 1e-6 * scale
            assert torch.allclose(g_sigma, ref_sigma, rtol=1e-5, atol=1e-7), (g_sigma, ref_sigma)


def test_schedule_change_needs_a_new_forward():
    W, H, F = 32, 16, 2
    zn, mesh, cams, sig, g_out = _inputs(W, H, F, seed=5)
    gbufs = [dhrs.GBuffer.from_arrays(zn[f], mesh[f]) for f in range(F)]
    gp = dhrs.SvgfParams(levels=2)
    sig_t = torch.from_numpy(_planes(sig).astype(np.float32)).cuda()
    gout_t = torch.from_numpy(_planes(g_out).astype(np.float32)).cuda()
    tape = dhrs.SvgfTape(W, H, F)
    tape.forward(gbufs, cams, sig_t, gp)
    tape.set_schedule(dhrs.TAPE_STORE)
    with pytest.raises(dhrs.DhrError):
        tape.backward(gbufs, cams, sig_t, gp, gout_t)
    with pytest.raises(dhrs.DhrError):
        tape.set_schedule(7)
    tape.forward(gbufs, cams, sig_t, gp)
    tape.backward(gbufs, cams, sig_t, gp, gout_t)
    torch.cuda.synchronize()


@pytest.mark.parametrize("F", [1, 2, 3])
def test_short_sequences_both_schedules(F):
    """One to three frames: the recomputing tape holds min(F, 2) slots and,
    for F <= 2, recomputes nothing; outputs bit-identical, gradients equal up
    to the atomics' order, and both match the oracle."""
    W, H = 40, 24
    zn, mesh, cams, sig, g_out = _inputs(W, H, F, seed=6)
    op = orc.SvgfParams(levels=3)
    out_o, gsig_o, gsigma_o = orc.svgf_seq_grad(zn, mesh, cams, sig, op, g_out)
    gbufs = [dhrs.GBuffer.from_arrays(zn[f], mesh[f]) for f in range(F)]
    gp = dhrs.SvgfParams(**op.__dict__)
    sig_t = torch.from_numpy(_planes(sig).astype(np.float32)).cuda()
    gout_t = torch.from_numpy(_planes(g_out).astype(np.float32)).cuda()
    res = []
    for sched in (dhrs.TAPE_RECOMPUTE, dhrs.TAPE_STORE):
        tape = dhrs.SvgfTape(W, H, F, sched)
        out = tape.forward(gbufs, cams, sig_t, gp)
        g_sig, g_sigma = tape.backward(gbufs, cams, sig_t, gp, gout_t)
        torch.cuda.synchronize()
        res.append((out, g_sig, g_sigma))
        per_frame = W * H * (16 * 2 + 8 * 3 + 16)
        assert tape.level_bytes(3) == per_frame * (min(F, 2) if sched == dhrs.TAPE_RECOMPUTE else F)
    assert torch.equal(res[0][0], res[1][0])
    assert float((res[0][1] - res[1][1]).abs().max()) <= 1e-6 * float(res[1][1].abs().max())
    g_sig = np.moveaxis(res[0][1].cpu().numpy(), 1, -1)
    assert np.abs(g_sig - gsig_o).max() <= 1e-3 * np.abs(gsig_o).max()
    assert np.abs(np.moveaxis(res[0][0].cpu().numpy(), 1, -1) - out_o).max() <= 1e-3


def test_level_records_grow_with_the_level_count():
    """A forward with more levels than the tape's records hold reallocates
    them; the backward then matches a fresh tape's."""
    W, H, F = 48, 32, 4
    zn, mesh, cams, sig, g_out = _inputs(W, H, F, seed=7)
    gbufs = [dhrs.GBuffer.from_arrays(zn[f], mesh[f]) for f in range(F)]
    sig_t = torch.from_numpy(_planes(sig).astype(np.float32)).cuda()
    gout_t = torch.from_numpy(_planes(g_out).astype(np.float32)).cuda()
    tape = dhrs.SvgfTape(W, H, F)
    p2, p5 = dhrs.SvgfParams(levels=2), dhrs.SvgfParams(levels=5)
    tape.forward(gbufs, cams, sig_t, p2)
    tape.backward(gbufs, cams, sig_t, p2, gout_t)
    out = tape.forward(gbufs, cams, sig_t, p5)
    g_sig, g_sigma = tape.backward(gbufs, cams, sig_t, p5, gout_t)
    fresh = dhrs.SvgfTape(W, H, F)
    out_f = fresh.forward(gbufs, cams, sig_t, p5)
    g_sig_f, g_sigma_f = fresh.backward(gbufs, cams, sig_t, p5, gout_t)
    torch.cuda.synchronize()
    assert torch.equal(out, out_f)
    assert float((g_sig - g_sig_f).abs().max()) <= 1e-6 * float(g_sig_f.abs().max())
    assert torch.allclose(g_sigma, g_sigma_f, rtol=1e-5, atol=1e-7)


def test_backward_on_a_caller_stream():
    """Forward and backward issued on a side stream of the caller's: after
    synchronising only that stream the gradients are complete (the tape's own
    streams join it before the call returns) and equal the default stream's."""
    W, H, F = 64, 40, 5
    zn, mesh, cams, sig, g_out = _inputs(W, H, F, seed=8)
    gbufs = [dhrs.GBuffer.from_arrays(zn[f], mesh[f]) for f in range(F)]
    gp = dhrs.SvgfParams()
    sig_t = torch.from_numpy(_planes(sig).astype(np.float32)).cuda()
    gout_t = torch.from_numpy(_planes(g_out).astype(np.float32)).cuda()
    ref = dhrs.SvgfTape(W, H, F)
    ref.forward(gbufs, cams, sig_t, gp)
    g_ref, s_ref = ref.backward(gbufs, cams, sig_t, gp, gout_t)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    tape = dhrs.SvgfTape(W, H, F)
    with torch.cuda.stream(side):
        tape.forward(gbufs, cams, sig_t, gp, stream=side)
        g_sig, g_sigma = tape.backward(gbufs, cams, sig_t, gp, gout_t, stream=side)
        host = (g_sig.to("cpu", non_blocking=False), g_sigma.to("cpu", non_blocking=False))
    side.synchronize()
    scale = float(g_ref.abs().max())
    assert float((host[0] - g_ref.cpu()).abs().max()) <= 1e-6 * scale
    assert torch.allclose(host[1], s_ref.cpu(), rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("W,H,F,levels", [(37, 23, 3, 5), (50, 31, 4, 8)])
def test_ragged_sizes_and_most_levels(W, H, F, levels):
    """Image sizes that cut the 32 x 8 tiles, and the largest level count
    (8: steps up to 128, beyond the image), under both record schedules,
    against the oracle's adjoint."""
    zn, mesh, cams, sig, g_out = _inputs(W, H, F, seed=9)
    op = orc.SvgfParams(levels=levels)
    out_o, gsig_o, gsigma_o = orc.svgf_seq_grad(zn, mesh, cams, sig, op, g_out)
    gbufs = [dhrs.GBuffer.from_arrays(zn[f], mesh[f]) for f in range(F)]
    gp = dhrs.SvgfParams(**op.__dict__)
    sig_t = torch.from_numpy(_planes(sig).astype(np.float32)).cuda()
    gout_t = torch.from_numpy(_planes(g_out).astype(np.float32)).cuda()
    for sched in (dhrs.TAPE_RECOMPUTE, dhrs.TAPE_STORE):
        tape = dhrs.SvgfTape(W, H, F, sched)
        out = tape.forward(gbufs, cams, sig_t, gp)
        g_sig, g_sigma = tape.backward(gbufs, cams, sig_t, gp, gout_t)
        torch.cuda.synchronize()
        out = np.moveaxis(out.cpu().numpy(), 1, -1)
        g_sig = np.moveaxis(g_sig.cpu().numpy(), 1, -1)
        g_sigma = g_sigma.cpu().numpy()
        assert np.abs(out - out_o).max() <= 1e-3
        assert np.abs(g_sig - gsig_o).max() <= 1e-3 * np.abs(gsig_o).max()
        for c in range(3):
            assert abs(g_sigma[c] - gsigma_o[c]) <= 1e-2 * abs(gsigma_o[c]) + 1e-4, (sched, c, g_sigma, gsigma_o)
