"""Serving form: continuous batching of many sessions (dhr_server_*) and the
delay reprojection (dhr_delay_warp, Section 4.1 / Fig. 5).

- dhr_delay_warp equals the oracle's warp on the oracle's own inputs.
- A session served by the batching server gives exactly what dhr_step_frame
  gives, alone and in a mix of sessions of other resolutions (same kernels,
  same per-pixel arithmetic: bit-identical, well inside 1e-3).
- Sessions of two sizes batched together equal the oracle's trace-then-filter
  frame by frame (no GPU path in between).
- Admission by device-memory budget, latest-wins request replacement.
"""
import numpy as np
import pytest

import oracle as orc
import paper_2406_06963_b300 as dhrs
import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_delay_warp_matches_oracle():
    s = wl.scene_boxes()
    S = orc.Scene(s)
    W, H = 160, 120
    cams = wl.orbit_path(6, W, H, degrees=12.0)
    cs, ct = cams[0], cams[5]
    zs, ms = orc.gbuffer_f32(orc.trace(S, cs, orc.TraceParams()), W, H)
    zt, mt = orc.gbuffer_f32(orc.trace(S, ct, orc.TraceParams()), W, H)
    r = np.random.default_rng(3)
    a = r.random((H, W)).astype(np.float32)
    b = r.random((H, W)).astype(np.float32)
    ra, rb, valid = orc.delay_warp(zt, mt, ct, zs, ms, cs, a.astype(np.float64), b.astype(np.float64))
    oa = torch.empty((H, W), device="cuda")
    ob = torch.empty_like(oa)
    dhrs.delay_warp(dhrs.GBuffer.from_arrays(zt, mt), ct, dhrs.GBuffer.from_arrays(zs, ms), cs,
                    torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), oa, ob)
    torch.cuda.synchronize()
    assert valid.mean() > 0.3 and (valid == 0).sum() > 0
    assert np.array_equal(oa.cpu().numpy(), ra.astype(np.float32))
    assert np.array_equal(ob.cpu().numpy(), rb.astype(np.float32))


def _run_server(sc, sessions, frames, budget=8 << 30, raster_min=None):
    """sessions: list of (W, H, path); returns outputs[session][frame].
    raster_min: sessions of at least this many pixels rasterise their primary
    visibility (None: the library's default, which these small sessions stay
    below, so they trace primary rays)."""
    srv = dhrs.Server(sc, budget)
    if raster_min is not None:
        srv.set_raster_min_pixels(raster_min)
    ids = [srv.open(w, h) for (w, h, _) in sessions]
    outs = {i: [] for i in range(len(sessions))}
    for f in range(frames):
        for k, (w, h, path) in enumerate(sessions):
            srv.submit(ids[k], path[f], f, dhrs.now_ns(), 1000 * k + f)
        assert srv.pump() == len(sessions)
        done = srv.poll(wait=True)
        while len([d for d in done if not d["dropped"]]) < len(sessions):
            done += srv.poll(wait=True)
        assert all(d["batch_size"] == len(sessions) for d in done)
        for k, (w, h, _) in enumerate(sessions):
            outs[k].append(srv.output(ids[k], w, h))
    return outs, srv


@pytest.mark.parametrize("raster_min", [None, 0, 20000])
def test_server_equals_step_frame_alone_and_in_mix(raster_min):
    """raster_min None: every session traces primary rays; 0: every session
    rasterises; 20000: a mix of both in one batch."""
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    A = (200, 120, wl.orbit_path(4, 200, 120, degrees=6.0))
    others = [(96, 64, wl.orbit_path(4, 96, 64, degrees=9.0, start_deg=40)),
              (333, 77, wl.orbit_path(4, 333, 77, degrees=3.0, start_deg=-30)),
              (64, 200, wl.orbit_path(4, 64, 200, degrees=5.0, start_deg=90))]
    alone, _ = _run_server(sc, [A], 4, raster_min=raster_min)
    mix, _ = _run_server(sc, others[:1] + [A] + others[1:], 4, raster_min=raster_min)
    sess = dhrs.Session(sc, 200, 120)
    a = torch.empty((120, 200), device="cuda")
    b = torch.empty_like(a)
    for f in range(4):
        sess.step(A[2][f], f, a, b)
        torch.cuda.synchronize()
        ref = (a.cpu().numpy(), b.cpu().numpy())
        for got in (alone[0][f], mix[1][f]):
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), f


@pytest.mark.parametrize("raster_min", [None, 0])
def test_server_sessions_match_oracle(raster_min):
    """Two sessions of different sizes batched together by the server, frame
    by frame against the oracle tracing the same poses itself and filtering
    them with orc_svgf_frame (Sections 3.1-3.3 and the serving form end to
    end, without the server-equals-session step in between).  The raw
    visibility of each pose (dhr_trace_visibility, the server's trace
    function) may differ from the oracle's only on rays the oracle flags as
    grazing; the filtered AO and shadow the server returns must be within
    1e-3 of the oracle's on every pixel whose filter footprint, over all
    frames so far, saw no such difference (a flipped bit spreads up to 62
    pixels through the levels and through the history)."""
    s = wl.scene_boxes()
    sc, S = dhrs.Scene(s), orc.Scene(s)
    sizes = [(256, 192, wl.orbit_path(5, 256, 192, degrees=10.0)),
             (160, 96, wl.orbit_path(5, 160, 96, degrees=8.0, start_deg=35))]
    outs, _ = _run_server(sc, sizes, 5, raster_min=raster_min)
    checked, total = 0, 0
    for k, (W, H, path) in enumerate(sizes):
        ost = orc.SvgfState(W, H)
        tainted = np.zeros((H, W), bool)
        for f, cam in enumerate(path):
            tr = orc.trace(S, cam, orc.TraceParams(frame=f))
            zn, mesh = orc.gbuffer_f32(tr, W, H)
            ref = ost.frame(zn, mesh, cam, tr["shadow_mask"].reshape(H, W), tr["ao_count"].reshape(H, W),
                            orc.SvgfParams())
            flagged = (tr["amb_primary"] | tr["amb_shadow"] | tr["amb_ao"]).reshape(H, W) > 0
            g = dhrs.GBuffer(W, H)
            m = torch.empty((H, W), dtype=torch.uint8, device="cuda")
            a = torch.empty_like(m)
            dhrs.trace_visibility(sc, cam, dhrs.TraceParams(frame=f), g, m, a)
            differ = (m.cpu().numpy() != tr["shadow_mask"].reshape(H, W)) | \
                     (a.cpu().numpy() != tr["ao_count"].reshape(H, W))
            assert not (differ & ~flagged).any(), (k, f)
            for y, x in zip(*np.nonzero(differ)):
                tainted[max(0, y - 72):y + 73, max(0, x - 72):x + 73] = True
            ok = ~tainted
            got_ao, got_sh = outs[k][f]
            e = np.maximum(np.abs(got_ao - ref["ao"]), np.abs(got_sh - ref["shadow"]))
            if ok.any():
                assert e[ok].max() <= 1e-3, (k, f, float(e[ok].max()))
            checked += int(ok.sum())
            total += W * H
    print(f"server vs oracle: {checked} of {total} pixel-frames checked")
    assert checked >= 0.8 * total


def test_server_admission_by_memory_budget():
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    need = dhrs.session_bytes(256, 256)
    srv = dhrs.Server(sc, 2 * need + need // 2)
    a = srv.open(256, 256)
    srv.open(256, 256)
    with pytest.raises(dhrs.DhrError) as e:
        srv.open(256, 256)
    assert e.value.status == 5
    small = srv.open(64, 64)              # a smaller session still fits
    srv.close_session(a)
    srv.open(256, 256)                    # memory freed: admitted
    st = srv.stats()
    assert st["open_sessions"] == 3 and st["used_bytes"] <= st["budget_bytes"]
    srv.close_session(small)


def test_server_session_closed_mid_flight():
    """A client that disconnects while its frame is in flight: the batch
    completes, the session's memory is released after it (not before), the
    request that was still queued for it is reported as dropped, and the
    other session of the batch is served as if alone."""
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    A = (128, 96, wl.orbit_path(3, 128, 96, degrees=6.0))
    B = (96, 64, wl.orbit_path(3, 96, 64, degrees=9.0, start_deg=40))
    alone, _ = _run_server(sc, [B], 2)
    srv = dhrs.Server(sc, 1 << 30)
    a, b = srv.open(A[0], A[1]), srv.open(B[0], B[1])
    used_two = srv.stats()["used_bytes"]
    srv.submit(a, A[2][0], 0, dhrs.now_ns(), 10)
    srv.submit(b, B[2][0], 0, dhrs.now_ns(), 20)
    assert srv.pump() == 2
    srv.submit(a, A[2][1], 1, dhrs.now_ns(), 11)      # queued behind the frame in flight
    srv.close_session(a)                              # disconnects mid-flight
    done = []
    while len(done) < 3:
        done += srv.poll(wait=True)
    by_id = {d["request_id"]: d for d in done}
    assert by_id[11]["dropped"] and not by_id[20]["dropped"]
    st = srv.stats()
    assert st["open_sessions"] == 1 and st["used_bytes"] < used_two
    got = srv.output(b, B[0], B[1])
    assert np.array_equal(got[0], alone[0][0][0]) and np.array_equal(got[1], alone[0][0][1])
    srv.submit(b, B[2][1], 1, dhrs.now_ns(), 21)      # the server goes on
    assert srv.pump() == 1
    done = srv.poll(wait=True)
    while not any(d["request_id"] == 21 for d in done):
        done += srv.poll(wait=True)
    got = srv.output(b, B[0], B[1])
    assert np.array_equal(got[0], alone[0][1][0]) and np.array_equal(got[1], alone[0][1][1])


def test_server_latest_request_wins():
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    path = wl.orbit_path(3, 64, 48)
    srv = dhrs.Server(sc, 1 << 30)
    sid = srv.open(64, 48)
    srv.submit(sid, path[0], 0, dhrs.now_ns(), 1)
    srv.submit(sid, path[1], 1, dhrs.now_ns(), 2)     # replaces request 1
    assert srv.pump() == 1
    done = srv.poll(wait=True)
    done += srv.poll(wait=True)
    by_id = {d["request_id"]: d for d in done}
    assert by_id[1]["dropped"] and not by_id[2]["dropped"]
    assert by_id[2]["t_done_ns"] >= by_id[2]["t_arrival_ns"]
    assert srv.stats()["dropped"] == 1


@pytest.mark.parametrize("raster_min", [None, 0])
def test_server_delay_warp_equals_components(raster_min):
    """A request with a target pose = trace + SVGF at the sent pose, then
    dhr_delay_warp onto a G-buffer of the target pose.  raster_min 0: the
    server rasterises both the traced pose's and the target pose's primary
    visibility (binned into the session's and the target's buffers)."""
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    W, H = 128, 96
    path = wl.orbit_path(8, W, H, degrees=14.0)
    srv = dhrs.Server(sc, 1 << 30)
    if raster_min is not None:
        srv.set_raster_min_pixels(raster_min)
    sid = srv.open(W, H)
    sess = dhrs.Session(sc, W, H)
    a = torch.empty((H, W), device="cuda")
    b = torch.empty_like(a)
    oa, ob = torch.empty_like(a), torch.empty_like(a)
    for f in range(4):
        tgt = path[f + 3]
        srv.submit(sid, path[f], f, dhrs.now_ns(), f, cam_target=tgt)
        srv.pump()
        srv.poll(wait=True)
        ga, gb = srv.output(sid, W, H)
        sess.step(path[f], f, a, b)
        gt = dhrs.GBuffer(W, H)
        m = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        dhrs.trace_visibility(sc, tgt, dhrs.TraceParams(frame=f), gt, m, m.clone())
        fb = sess.frame_buffers()
        gs = dhrs.GBuffer(W, H)
        gs.depth_normal.copy_(dhrs.device_copy(fb["depth_normal"], (H, W, 4), "float32"))
        gs.mesh.copy_(dhrs.device_copy(fb["mesh"], (H, W), "int32"))
        dhrs.delay_warp(gt, tgt, gs, path[f], a, b, oa, ob)
        torch.cuda.synchronize()
        assert np.array_equal(ga, oa.cpu().numpy()) and np.array_equal(gb, ob.cpu().numpy()), f
        assert float((ga == 1).mean()) < 0.9


def test_server_batch_pixel_cap():
    """A batch takes sessions in request order until the next would pass the
    pixel cap (at least one); cap 0 takes every ready session."""
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    W = H = 1024
    path = wl.orbit_path(2, W, H)
    for cap, expect in ((2 * W * H, [2, 1]), (W * H - 1, [1, 1]), (0, [3])):
        srv = dhrs.Server(sc, 8 << 30)
        srv.set_max_batch_pixels(cap)
        ids = [srv.open(W, H) for _ in range(3)]
        for k, sid in enumerate(ids):
            srv.submit(sid, path[0], 0, dhrs.now_ns(), k)
        launched = [srv.pump(), srv.pump()]
        assert [n for n in launched if n] == expect[:2], (cap, launched)
        done = []
        while len(done) < 3:
            done += srv.poll(wait=True)
            if len(done) < 3:
                n = srv.pump()
                assert n in (0, 1)
        assert sum(1 for d in done if not d["dropped"]) == 3
        assert max(d["batch_size"] for d in done) == max(expect)


# ----------------------------------------------------------------------------
# the device-resident request loop (dhr_server_loop_*)
# ----------------------------------------------------------------------------
@pytest.fixture(autouse=False)
def no_gc():
    """While a device loop runs, a device-wide synchronisation anywhere in the
    process (here: cudaFree or cudaFreeHost from a garbage-collected scene or
    server of an earlier test) would wait for the loop to end; collect first
    and keep the collector off meanwhile."""
    import gc
    gc.collect()
    gc.disable()
    yield
    gc.enable()

def _collect(srv, want, limit_s=30.0):
    """Poll until `want` requests are reported (completed or dropped)."""
    import time
    got, t0 = [], time.perf_counter()
    while len(got) < want:
        got += srv.poll(wait=True)
        assert time.perf_counter() - t0 < limit_s, got
    return got


@pytest.mark.parametrize("raster_min", [None, 20000])
def test_device_loop_equals_host_batches(no_gc, raster_min):
    """The same per-session request sequences through the device loop and
    through host-formed batches give bit-identical outputs (same kernels,
    same inputs, whatever the batching; raster_min 20000: the two larger
    sessions rasterise, with raster constants formed on the device by the
    loop and on the host for the host batches)."""
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    sessions = [(200, 120, wl.orbit_path(4, 200, 120, degrees=6.0)),
                (96, 64, wl.orbit_path(4, 96, 64, degrees=9.0, start_deg=40)),
                (333, 77, wl.orbit_path(4, 333, 77, degrees=3.0, start_deg=-30))]
    # the host-batched server stays referenced: destroying it frees pinned
    # memory, a device-wide synchronisation that would wait for the loop
    host, host_srv = _run_server(sc, sessions, 4, raster_min=raster_min)
    srv = dhrs.Server(sc, 8 << 30)
    if raster_min is not None:
        srv.set_raster_min_pixels(raster_min)
    ids = [srv.open(w, h) for (w, h, _p) in sessions]
    srv.loop_start(idle_ms=5000, max_run_ms=60000)
    for f in range(4):
        for k, (w, h, path) in enumerate(sessions):
            srv.submit(ids[k], path[f], f, dhrs.now_ns(), 1000 * k + f)
        done = _collect(srv, len(sessions))
        assert not any(d["dropped"] for d in done)
        assert sorted(d["request_id"] for d in done) == sorted(1000 * k + f for k in range(len(sessions)))
        assert all(d["t_done_ns"] >= d["t_start_ns"] >= d["t_arrival_ns"] - 1_000_000 for d in done)
        for k, (w, h, _p) in enumerate(sessions):
            a, b = srv.output(ids[k], w, h)
            assert np.array_equal(a, host[k][f][0]) and np.array_equal(b, host[k][f][1])
    running, passes = srv.loop_status()
    assert running and passes > 0
    srv.loop_stop()
    assert not srv.loop_status()[0]


def test_device_loop_delay_warp_equals_host_batches(no_gc):
    """Requests with target poses, every session rasterising both poses:
    the device loop (raster constants of both poses formed on the device)
    and host-formed batches give bit-identical warped outputs."""
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    sessions = [(200, 120, wl.orbit_path(7, 200, 120, degrees=6.0)),
                (96, 64, wl.orbit_path(7, 96, 64, degrees=9.0, start_deg=40))]
    outs = {}
    keep = []
    for mode in ("host", "loop"):
        srv = dhrs.Server(sc, 4 << 30)
        keep.append(srv)   # destroying a server synchronises the device: not while a loop runs
        srv.set_raster_min_pixels(0)
        ids = [srv.open(w, h) for (w, h, _p) in sessions]
        if mode == "loop":
            srv.loop_start(idle_ms=5000, max_run_ms=60000)
        res = []
        for f in range(4):
            for k, (w, h, path) in enumerate(sessions):
                srv.submit(ids[k], path[f], f, dhrs.now_ns(), 1000 * k + f, cam_target=path[f + 3])
            if mode == "host":
                srv.pump()
                done = srv.poll(wait=True)
                while len([d for d in done if not d["dropped"]]) < len(sessions):
                    done += srv.poll(wait=True)
            else:
                _collect(srv, len(sessions))
            res.append([srv.output(ids[k], w, h) for k, (w, h, _p) in enumerate(sessions)])
        if mode == "loop":
            srv.loop_stop()
        outs[mode] = res
    for f in range(4):
        for k in range(len(sessions)):
            for c in range(2):
                assert np.array_equal(outs["host"][f][k][c], outs["loop"][f][k][c]), (f, k, c)
        assert float((outs["host"][f][0][0] == 1).mean()) < 0.9


def test_device_loop_times_out_when_work_is_withheld(no_gc):
    """No request arrives: the loop's bounded wait runs out after its idle
    limit, it ends by itself, and the host sees DHR_ERR_TIMEOUT from poll
    and from loop_stop; the context stays usable and the host-driven mode
    serves the session afterwards."""
    import time
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    srv = dhrs.Server(sc, 1 << 30)
    sid = srv.open(64, 48)
    srv.loop_start(idle_ms=100, max_run_ms=20000)
    t0 = time.perf_counter()
    with pytest.raises(dhrs.DhrError) as e:
        srv.poll(wait=True)
    assert e.value.status == 4
    assert time.perf_counter() - t0 < 10.0
    running, passes = srv.loop_status()
    assert not running and passes > 0
    with pytest.raises(dhrs.DhrError) as e:
        srv.loop_stop()
    assert e.value.status == 4
    cam = wl.boxes_camera(64, 48)
    srv.submit(sid, cam, 0, dhrs.now_ns(), 7)
    assert srv.pump() == 1
    done = _collect(srv, 1)
    assert done[0]["request_id"] == 7 and not done[0]["dropped"]
    a, _ = srv.output(sid, 64, 48)
    assert np.isfinite(a).all()


def test_device_loop_latest_wins_and_accounts_every_request(no_gc):
    """Bursts of requests per session while the loop runs: every request is
    reported exactly once; a dropped request is always older than a
    completed one of its session; the newest request of every session
    completes.  Sessions closed while the loop runs are released."""
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    srv = dhrs.Server(sc, 8 << 30)
    sizes = [(128, 96), (256, 160), (64, 64), (200, 100)]
    ids = [srv.open(w, h) for (w, h) in sizes]
    paths = [wl.orbit_path(12, w, h, degrees=10.0, start_deg=20 * k) for k, (w, h) in enumerate(sizes)]
    srv.loop_start(idle_ms=5000, max_run_ms=60000)
    rid = 0
    sent = {}
    for f in range(12):
        for k in range(len(sizes)):
            srv.submit(ids[k], paths[k][f], f, dhrs.now_ns(), rid)
            sent[rid] = k
            rid += 1
    done = _collect(srv, rid)
    assert sorted(d["request_id"] for d in done) == list(range(rid))
    for k in range(len(sizes)):
        mine = [d for d in done if sent[d["request_id"]] == k]
        completed = [d["request_id"] for d in mine if not d["dropped"]]
        assert max(d["request_id"] for d in mine) in completed
        for d in mine:
            if d["dropped"]:
                assert any(c > d["request_id"] for c in completed)
    before = srv.stats()["used_bytes"]
    srv.close_session(ids[1])
    srv.submit(ids[0], paths[0][0], 99, dhrs.now_ns(), rid)
    _collect(srv, 1)
    srv.pump()
    srv.loop_stop()
    assert srv.stats()["used_bytes"] == before - dhrs.session_bytes(*sizes[1])
