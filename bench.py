"""Benchmark of the DHR+S server hot path on one B300 (or N replicas).

One step = one frame of the hot path through dhr_step_frame: LBVH traversal
of the primary G-buffer rays, one cone-jittered shadow ray and one
cosine-weighted AO ray per foreground pixel, then the modified SVGF
(temporal accumulation + variance + 5 a-trous levels) at 1920x1080 on the
776,050-triangle terrain scene, frames taken from the 60-frame seeded camera
spline.  The scene and BVH are built once before timing (static scene).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (brute
force, fp64) on a bounded pixel sample per step on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mrays/s; ms/frame (trace+SVGF) at 1080p; p99 frame latency at 32 clients"
W, H = 1920, 1080
N_FRAMES = 60
L2_FLUSH_BYTES = 256 << 20
WORKLOAD = "terrain776k_1080p_spline60"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


# sources each profiled kernel is compiled from
KERNEL_SOURCES = {
    "trace_kernel": ["trace.cu", "trace_device.cuh", "sampling.cuh", "common.cuh"],
    "trace_kernel_raster_form": ["trace.cu", "trace_device.cuh", "sampling.cuh", "common.cuh"],
    "atrous_kernel": ["svgf.cu", "svgf_kernels.cuh", "common.cuh"],
    "temporal_kernel": ["svgf.cu", "svgf_kernels.cuh", "common.cuh"],
    "atrous_bwd_a": ["svgf_adjoint.cu", "svgf_kernels.cuh", "common.cuh"],
    "atrous_bwd_b": ["svgf_adjoint.cu", "svgf_kernels.cuh", "common.cuh"],
    "temporal_bwd_kernel": ["svgf_adjoint.cu", "svgf_kernels.cuh", "common.cuh"],
}


def csrc_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2406_06963_b300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel's sources changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            t = json.load(f)
    except OSError:
        return None
    e = t.get(kernel)
    if not e or e.get("csrc_sha") != csrc_hash(kernel):
        return None
    return e.get("dram_bytes_per_launch")


def _ncu_field(kernel: str, field: str):
    """Another figure of the committed capture of `kernel` (None when the
    kernel's sources changed since)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            e = json.load(f).get(kernel)
    except OSError:
        return None
    if not e or e.get("csrc_sha") != csrc_hash(kernel):
        return None
    return e.get(field)


def _svgf_traffic():
    """DRAM bytes of one frame's SVGF (temporal + 5 a-trous launches) from the
    committed captures, or None when either kernel changed since."""
    t, a = _traffic("temporal_kernel"), _traffic("atrous_kernel")
    return None if t is None or a is None else t + 5 * a


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


from paper_2406_06963_b300.replicas import barrier as _barrier  # noqa: E402
from paper_2406_06963_b300.replicas import dist_env as _dist  # noqa: E402
from paper_2406_06963_b300.replicas import job_throughput, max_over_ranks  # noqa: E402


def bench_config(ws, n_triangles):
    """The workload of one step, the same for both arms."""
    return {"workload": WORKLOAD, "resolution": [W, H], "triangles": int(n_triangles),
            "frames_in_path": N_FRAMES, "spp": {"shadow": 1, "ao": 1}, "svgf_levels": 5,
            "alpha": 0.2, "parallelism": f"replicas{ws}",
            "l2": "no flush: per-frame working set (BVH 87 MB + G-buffers + SVGF buffers, > 300 MB) "
                  "exceeds the 126 MB L2; stage split flushed (256 MB write) before every frame",
            "pipelining": "frame i + 1 traced while frame i is filtered (session streams)"}


def run_ours(args):
    import torch

    import paper_2406_06963_b300 as dhrs
    import workloads as wl

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    scene_d = wl.scene_terrain()
    cams = wl.spline_path(scene_d["terrain"], N_FRAMES, W, H)
    stream = torch.cuda.current_stream()
    sc = dhrs.Scene(scene_d)
    info = sc.info()
    primary = dhrs.PRIMARY_RASTER if args.primary == "raster" else dhrs.PRIMARY_TRAVERSE
    tp = dhrs.TraceParams(ao_spp=1, primary=primary)
    sp = dhrs.SvgfParams(ao_spp=1, levels=5, alpha=0.2)
    sess = dhrs.Session(sc, W, H, dhrs.DHR_FP32, tp, sp)
    ao_out = torch.empty((H, W), device="cuda")
    sh_out = torch.empty((H, W), device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    K, Wm = args.steps, args.warmup
    for i in range(Wm):
        sess.step(cams[i % N_FRAMES], i, ao_out, sh_out)
    torch.cuda.synchronize()

    # timed region: K consecutive frames through the session (frame i + 1's
    # trace overlaps frame i's filter), timed as a whole with events on the
    # stream; no L2 flush between frames -- the per-frame working set (BVH
    # 87 MB, G-buffers 2 x 41 MB, SVGF buffers ~240 MB at 1080p) is larger
    # than the 126 MB L2
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    _barrier(ws)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    e0.record(stream)
    for i in range(K):
        sess.step(cams[(Wm + i) % N_FRAMES], Wm + i, ao_out, sh_out)
    e1.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    t_wall = time.perf_counter() - t_wall
    own_ms = e0.elapsed_time(e1)

    # stage split: the same frames through the two component calls
    g = dhrs.GBuffer(W, H)
    gp = dhrs.GBuffer(W, H)
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    aoc = torch.empty_like(mask)
    st = dhrs.SvgfState(W, H)
    tr_ms, sv_ms = [], []
    prev_cam = None
    for i in range(-Wm, K):     # Wm untimed frames first, so the history is warm
        f = (Wm + i) % N_FRAMES
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        flush.fill_(float(i))
        e0.record(stream)
        # the traversal form: one kernel with all three ray types (the roofline's kernel)
        dhrs.trace_visibility(sc, cams[f], dhrs.TraceParams(ao_spp=1, frame=Wm + i,
                                                            primary=dhrs.PRIMARY_TRAVERSE), g, mask, aoc)
        e1.record(stream)
        st.reconstruct(g, gp if prev_cam is not None else None, cams[f], prev_cam, mask, aoc, sp, ao_out, sh_out)
        e2.record(stream)
        torch.cuda.synchronize()
        if i >= 0:
            tr_ms.append(e0.elapsed_time(e1))
            sv_ms.append(e1.elapsed_time(e2))
        g, gp = gp, g
        prev_cam = cams[f]
    # the trace call in the session's form (rasterised primary visibility by
    # default), timed on the device in two parts: primary pre-pass, trace kernel
    tr_sess_ms, tr_pre_ms, tr_ker_ms = [], [], []
    for i in range(K):
        flush.fill_(float(i))
        pre, ker = dhrs.trace_timed(sc, cams[(Wm + i) % N_FRAMES],
                                    dhrs.TraceParams(ao_spp=1, frame=Wm + i, primary=primary), g, mask, aoc)
        tr_pre_ms.append(pre)
        tr_ker_ms.append(ker)
        tr_sess_ms.append(pre + ker)
    clk = clocks.stop()

    # end to end through the host-output entry point (camera in, filtered AO and
    # shadow out to pinned host memory every step)
    # (streaming form: frame i's copy to pinned host memory overlaps the next
    # frames; a frame's result is waited for two frames later, before its
    # host buffers are reused)
    hbuf = [(torch.empty((H, W), pin_memory=True), torch.empty((H, W), pin_memory=True)) for _ in range(3)]
    sess2 = dhrs.Session(sc, W, H, dhrs.DHR_FP32, tp, sp)
    for i in range(Wm):
        sess2.step_host(cams[i % N_FRAMES], i, *hbuf[0])
    _barrier(ws)
    t0 = time.perf_counter()
    tickets = []
    for i in range(K):
        tickets.append(sess2.step_host_async(cams[(Wm + i) % N_FRAMES], Wm + i, *hbuf[i % 3]))
        if i >= 2:
            sess2.wait(tickets[i - 2])   # frame i - 2 is in host memory
    for t in tickets[-2:]:
        sess2.wait(t)
    e2e_own_s = time.perf_counter() - t0

    # transport: the last frame's raw trace outputs, packed losslessly
    fb = sess.frame_buffers()
    m_last = dhrs.device_copy(fb["mask"], (H, W), "uint8")
    a_last = dhrs.device_copy(fb["ao"], (H, W), "uint8")
    pack_ms = []
    for _ in range(11):   # median of 10 after one warm-up call (host jitter enters through the readback)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record()
        packed = dhrs.pack_visibility(m_last, a_last, 1, 1)
        p1.record()
        torch.cuda.synchronize()
        pack_ms.append(p0.elapsed_time(p1))
    transport = {"raw_bytes_per_frame": 2 * W * H, "packed_bytes_per_frame": packed.numel() * 4,
                 "pack_ms_incl_size_readback": round(statistics.median(pack_ms[1:]), 4),
                 "format": "bit planes x 32x8 tiles, uniform tiles 2 bits (dhr_visibility_pack)"}

    # rays and traversal work of every frame of the path (counting variant of
    # the trace kernel, run after the timed regions)
    stats = [dhrs.trace_stats(sc, cams[f], dhrs.TraceParams(ao_spp=1, frame=f, primary=dhrs.PRIMARY_TRAVERSE))
             for f in range(N_FRAMES)]
    # the session form's work (rasterised primaries: tile-list tests; only
    # traversed tiles visit nodes)
    stats_s = stats if primary == dhrs.PRIMARY_TRAVERSE else \
        [dhrs.trace_stats(sc, cams[f], dhrs.TraceParams(ao_spp=1, frame=f, primary=primary)) for f in range(N_FRAMES)]
    rays = [sum(s["rays"]) for s in stats]
    sec_rays = [s["rays"][1] + s["rays"][2] for s in stats]
    step_rays = sum(rays[(Wm + i) % N_FRAMES] for i in range(K))
    step_sec = sum(sec_rays[(Wm + i) % N_FRAMES] for i in range(K))
    # whole job: rays of all ranks / the slowest rank's time
    value, job_rays, total_s = job_throughput(ws, step_rays, own_ms * 1e-3)
    value /= 1e6
    total_ms = total_s * 1e3
    e2e_value, _, e2e_s = job_throughput(ws, step_rays, e2e_own_s)
    e2e_value /= 1e6
    job_sec = ws * step_sec if ws == 1 else job_throughput(ws, step_sec, 1.0)[1]

    peaks, peak_src = _peaks()
    trace_ms = statistics.mean(tr_ms)
    svgf_ms = statistics.mean(sv_ms)
    # dominant kernel: trace.  Algorithmic work per frame from the counting
    # variant: a node visit is two slab tests (24 fp32 lane-ops) and fetches
    # one 64-byte node, a triangle test is one watertight test (30 lane-ops)
    # on 36 bytes of vertices.  Held against the fp32 lane-op rate and the
    # measured L2 read bandwidth; the larger fraction is the roofline's.
    sub = [(Wm + i) % N_FRAMES for i in range(K)]
    visits = statistics.mean(sum(stats[f]["visits"]) for f in sub)
    tests = statistics.mean(sum(stats[f]["tests"]) for f in sub)
    alu_peak = 148 * 128 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12   # lane-ops/s, Tops
    l2_gbs = dhrs.l2_read_bandwidth()

    def work(st_list, types, prim_hits=False):
        """(lane-ops, bytes) per frame over the frames timed; prim_hits: the
        primary rays counted as one closest-hit triangle test per foreground
        pixel (rasterised primaries: the binning candidates that miss their
        pixel are not the method's work)."""
        ops, byt = [], []
        for f in sub:
            v = sum(st_list[f]["visits"][i] for i in types)
            t = sum(st_list[f]["tests"][i] for i in types)
            if prim_hits:
                t += st_list[f]["rays"][2]          # foreground pixels (one AO ray each)
            ops.append(24 * v + 30 * t)
            byt.append(64 * v + 36 * t)
        return statistics.mean(ops), statistics.mean(byt)

    def roof(ops, byt, ms):
        a_alu = ops / (ms * 1e-3) / 1e12
        a_l2 = byt / (ms * 1e-3) / 1e9
        f_alu, f_l2 = a_alu / alu_peak, a_l2 / l2_gbs
        return {"bound": "l2" if f_l2 >= f_alu else "alu",
                "achieved": round(a_l2 if f_l2 >= f_alu else a_alu, 3),
                "peak": round(l2_gbs if f_l2 >= f_alu else alu_peak, 2),
                "unit": "GB/s" if f_l2 >= f_alu else "Tops/s (fp32 lane ops)",
                "frac": round(max(f_alu, f_l2), 4),
                "alu": {"achieved": round(a_alu, 3), "peak": round(alu_peak, 2), "unit": "Tops/s (fp32 lane ops)",
                        "frac": round(f_alu, 4)},
                "l2": {"achieved": round(a_l2, 1), "peak": round(l2_gbs, 1), "unit": "GB/s", "frac": round(f_l2, 4)}}

    # the traversal form: all three ray types traversed (stage split)
    ops_t, byt_t = work(stats, (0, 1, 2))
    # the session's trace kernel: rasterised primaries (one closest-hit test
    # per foreground pixel), shadow and AO rays traversed
    raster = primary == dhrs.PRIMARY_RASTER
    ops_s, byt_s = work(stats_s, (1, 2), prim_hits=True) if raster else (ops_t, byt_t)
    kernel_s = ("trace_kernel<0, 0, 1> (rasterised primary visibility + shadow + AO rays)" if raster
                else "trace_kernel<0, 0, 0> (primary + shadow + AO rays)")
    ker_ms = statistics.mean(tr_ker_ms)
    traffic_key = "trace_kernel_raster_form" if raster else "trace_kernel"
    # the counts a first version reported: 36 lane-ops per visit, 48 per
    # test, every tile-list candidate a test
    ops_b = statistics.mean(sum(stats_s[f]["visits"]) * 36 + sum(stats_s[f]["tests"]) * 48 for f in sub)
    svgf_bpp = 358        # per pixel: temporal 106 + 5 levels x 52 - 8 (the last writes no variance)
    svgf_gbs = W * H * svgf_bpp / (svgf_ms * 1e-3) / 1e9
    res = {
        "metric": METRIC, "value": round(value, 2), "unit": "Mrays/s", "n_gpus": ws, "steps": K,
        "warmup": Wm, "ms_per_step": round(total_ms / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(ws, info["n_triangles"]),
        "primary_visibility": args.primary,
        "ms_per_frame": {"trace_svgf": round(total_ms / K, 4), "trace": round(trace_ms, 4),
                         "trace_session_form": round(statistics.mean(tr_sess_ms), 4),
                         "trace_session_form_parts": {"primary_prepass": round(statistics.mean(tr_pre_ms), 4),
                                                      "trace_kernel": round(ker_ms, 4)},
                         "svgf": round(svgf_ms, 4)},
        "secondary_mrays_s": round(job_sec / (total_ms * 1e-3) / 1e6, 2),
        "rays_per_frame": round(step_rays / K),
        "bvh": {"height": info["height"], "build_ms": round(info["build_ms"], 3),
                "visits_per_ray": round(visits / (step_rays / K), 2),
                "tests_per_ray": round(tests / (step_rays / K), 2),
                # per ray type {primary, shadow, AO}, over all frames of the path
                "by_type": {t: {"rays_per_frame": round(sum(st["rays"][i] for st in stats) / N_FRAMES),
                                "visits_per_ray": round(sum(st["visits"][i] for st in stats)
                                                        / max(1, sum(st["rays"][i] for st in stats)), 2),
                                "tests_per_ray": round(sum(st["tests"][i] for st in stats)
                                                       / max(1, sum(st["rays"][i] for st in stats)), 2)}
                            for i, t in enumerate(("primary", "shadow", "ao"))}},
        # dominant kernel of the session frames (the headline's path), timed
        # alone after an L2 flush through dhr_trace_timed
        "roofline": {"kernel": kernel_s, **roof(ops_s, byt_s, ker_ms), "traffic": _traffic(traffic_key),
                     "work_per_frame": {"lane_ops": round(ops_s), "bytes": round(byt_s),
                                        "counts": "24 lane-ops + 64 B per node visit, 30 lane-ops + 36 B per "
                                                  "triangle test; rasterised primaries: one test per "
                                                  "foreground pixel"},
                     "peak_source": {"alu": "148 SMs x 128 fp32 lanes x max SM clock (%s)" % peak_src,
                                     "l2": "dhr_l2_read_bandwidth: 48 MB L2-resident buffer read 40 times "
                                           "with L2-only loads, this run"},
                     # first version's count (36 / 48 lane-ops, every tile-list candidate a test)
                     "builder_count_frac_alu": round(ops_b / (ker_ms * 1e-3) / 1e12 / alu_peak, 4),
                     # the limiters ncu measures for this kernel (committed capture):
                     # instruction issue and the L1/tex pipe (node fetches, local stack)
                     "ncu_issue_active_pct": _ncu_field(traffic_key, "issue_active_pct"),
                     "ncu_l1tex_throughput_pct": _ncu_field(traffic_key, "l1tex_throughput_pct"),
                     "ncu_l2_throughput_pct": _ncu_field(traffic_key, "lts_throughput_pct")},
        # the same kernel with traversed primaries (all three ray types), stage split
        "roofline_traversal_form": {"kernel": "trace_kernel<0, 0, 0>", **roof(ops_t, byt_t, trace_ms),
                                    "traffic": _traffic("trace_kernel")},
        "roofline_svgf": {"bound": "hbm", "achieved": round(svgf_gbs, 1), "peak": peaks["hbm_gbs"],
                          "unit": "GB/s", "frac": round(svgf_gbs / peaks["hbm_gbs"], 4),
                          "algorithmic_bytes_per_px": svgf_bpp, "peak_source": peak_src,
                          "traffic_per_frame": _svgf_traffic()},
        "e2e": {"value": round(e2e_value, 2), "unit": "Mrays/s", "h2d_bytes_per_step": 60,
                "d2h_bytes_per_step": 2 * 4 * W * H,
                "ms_per_step": round(e2e_s * 1e3 / K, 4)},
        "transport": transport,
        # per session frame: trace (+ tile-count clear, binning and big-triangle
        # binning when rasterised), temporal, 5 a-trous levels
        "gpu_launches": (10 if primary == dhrs.PRIMARY_RASTER else 7) * K,
        "clocks": clk,
        "wall_s_timed_region": round(t_wall, 3),
    }
    if not args.no_forms:
        res["serving"] = run_serving(sc, scene_d, seconds=args.serve_seconds)
        res["serving_device_loop"] = run_serving(sc, scene_d, seconds=args.serve_seconds, mode="device_loop")
        res["precision_form"] = run_precision_form(sc, scene_d)
        res["adjoint"] = run_adjoint(sc, scene_d)
        res["denoise_variants"] = run_denoise_variants(sc, scene_d)
        res["selective_shadows"] = run_selective(sc, scene_d)
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(scene_d, cams, sample_px=args.cpu_pixels,
                                           rays_per_frame=res["rays_per_frame"])
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return res if rank == 0 else None


# pixel cap of one serving batch (dhr_server_set_max_batch_pixels; 0 = none;
# the library default is 2^21)
SERVE_BATCH_PX = int(os.environ.get("DHR_SERVE_BATCH_PX", str(2 << 20)))


def run_serving(sc, scene_d, seconds=10.0, n_sessions=32, budget=64 << 30, max_batch_px=SERVE_BATCH_PX,
                mode="host"):
    """32 thin-client sessions, resolutions drawn from {640x360, 1280x720,
    1920x1080, 2560x1440}, each sending camera poses as a 60 Hz Poisson
    process along its own seeded spline, with a network delay U[0, 200] ms
    per session (the request arrives late and its result is warped to the
    pose at arrival).  Real-time simulation for `seconds`; latency = device
    completion - arrival at the server (network delay excluded).
    mode "host": the host forms each batch (dhr_server_pump); "device_loop":
    the device-resident request loop (dhr_server_loop_start) takes the
    requests from its mailboxes and forms the batches itself."""
    import gc

    import numpy as np

    import paper_2406_06963_b300 as dhrs
    import workloads as wl
    r = wl.rng_for(4)
    sizes = [(640, 360), (1280, 720), (1920, 1080), (2560, 1440)]
    srv = dhrs.Server(sc, budget)
    srv.set_max_batch_pixels(max_batch_px)
    n_poses = int((seconds + 0.3) * 60) + 2
    events, refused, admitted, px_of = [], 0, 0, {}
    for k in range(n_sessions):
        w, h = sizes[int(r.integers(0, 4))]
        d = float(r.uniform(0.0, 0.2))
        try:
            sid = srv.open(w, h)
        except dhrs.DhrError as e:
            if e.status != 5:
                raise
            refused += 1
            continue
        admitted += 1
        px_of[sid] = w * h
        path = wl.spline_path(scene_d["terrain"], n_poses, w, h, index=4, stream=k)
        t = float(r.exponential(1 / 60))
        i = 0
        while t < seconds:
            fi = min(int(round(t * 60)), n_poses - 1)
            ti = min(int(round((t + d) * 60)), n_poses - 1)
            events.append((t + d, sid, path[fi], path[ti] if ti != fi else None, i))
            t += float(r.exponential(1 / 60))
            i += 1
    events.sort(key=lambda e: e[0])
    lat, done_px, batches = [], 0, []
    dropped = 0
    if mode == "device_loop":
        # no device-wide synchronisation while the loop runs (a collected
        # CUDA object would make one)
        gc.collect()
        gc.disable()
        srv.loop_start(idle_ms=2000, max_run_ms=int((seconds + 30) * 1000))
    start = dhrs.now_ns() + 20_000_000
    idx = 0
    rid = 0
    while True:
        now = (dhrs.now_ns() - start) * 1e-9
        while idx < len(events) and events[idx][0] <= now:
            ta, sid, cam, tgt, fr = events[idx]
            srv.submit(sid, cam, fr, start + int(ta * 1e9), rid, cam_target=tgt)
            rid += 1
            idx += 1
        srv.pump()
        for c in srv.poll(wait=idx >= len(events)):
            if c["dropped"]:
                dropped += 1
                continue
            lat.append((c["t_done_ns"] - c["t_arrival_ns"]) * 1e-6)
            done_px += px_of[c["session"]]
            batches.append(c["batch_size"])
        if idx >= len(events) and len(lat) + dropped >= len(events):
            break
    wall = (dhrs.now_ns() - start) * 1e-9
    if mode == "device_loop":
        srv.loop_stop()
        gc.enable()
    st = srv.stats()
    srv.close()
    lat = np.array(lat)
    return {"workload": "32 sessions x 60 Hz Poisson, delay U[0,200] ms, terrain776k", "mode": mode,
            "sessions_admitted": admitted, "sessions_refused": refused, "requests": len(events),
            "completed": int(len(lat)), "dropped_latest_wins": dropped,
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "frames_per_s": round(len(lat) / wall, 1), "mpx_per_s": round(done_px / wall / 1e6, 1),
            "mean_batch": round(float(np.mean(batches)), 2), "batches": int(st["batches"]),
            "max_batch_pixels": max_batch_px,
            "device_bytes": int(st["used_bytes"]) if st["open_sessions"] else None, "seconds": round(wall, 3)}


def run_precision_form(sc, scene_d, frames=10, warm=3):
    """Same scene and path at 3840x2160: FP16-storage form vs FP32 path."""
    import numpy as np
    import torch

    import paper_2406_06963_b300 as dhrs
    import workloads as wl
    W4, H4 = 3840, 2160
    cams = wl.spline_path(scene_d["terrain"], N_FRAMES, W4, H4)
    res = {}
    outs = {}
    for name, prec in (("fp32", dhrs.DHR_FP32), ("fp16", dhrs.DHR_FP16)):
        sess = dhrs.Session(sc, W4, H4, prec)
        a = torch.empty((H4, W4), device="cuda")
        b = torch.empty_like(a)
        for i in range(warm):
            sess.step(cams[i], i, a, b)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(warm, warm + frames):
            sess.step(cams[i], i, a, b)
        e1.record()
        torch.cuda.synchronize()
        res[name + "_ms_per_frame"] = round(e0.elapsed_time(e1) / frames, 4)
        outs[name] = torch.stack([a, b]).clone()
        sess.close()
    e = (outs["fp16"] - outs["fp32"]).abs().flatten().cpu().numpy()
    res["fp16_vs_fp32_abs_err"] = {"max": float(e.max()), "p99": float(np.percentile(e, 99)),
                                   "mean": float(e.mean())}
    res["workload"] = "terrain776k_3840x2160"
    return res


def run_adjoint(sc, scene_d, frames=8, W=1280, H=720, fit_steps=4):
    """Differentiable SVGF over 8 frames at 1280x720: forward + backward
    time, L2 loss against a 255-spp AO reference, a few Adam steps on
    log(sigma_z, sigma_n, sigma_l)."""
    import torch

    import paper_2406_06963_b300 as dhrs
    import workloads as wl
    cams = wl.spline_path(scene_d["terrain"], N_FRAMES, W, H)[:frames]
    gbufs, sig, ref = [], [], []
    for f, cam in enumerate(cams):
        g = dhrs.GBuffer(W, H)
        m = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        a = torch.empty_like(m)
        dhrs.trace_visibility(sc, cam, dhrs.TraceParams(ao_spp=1, frame=f), g, m, a)
        gbufs.append(g)
        sig.append(torch.stack([a.float(), (m & 1).float()]))
        g2 = dhrs.GBuffer(W, H)
        a2 = torch.empty_like(m)
        dhrs.trace_visibility(sc, cam, dhrs.TraceParams(ao_spp=255, frame=f), g2, m.clone(), a2)
        ref.append(a2.float() / 255.0)
    sig = torch.stack(sig).contiguous()
    ref = torch.stack(ref)
    p = dhrs.SvgfParams()
    g_out = torch.zeros_like(sig)

    def time_fb(tape, reps=3):
        """median forward and backward times (ms) of `reps` runs after one warm-up"""
        out = tape.forward(gbufs, cams, sig, p)
        g_out[:, 0] = 2 * (out[:, 0] - ref)
        tape.backward(gbufs, cams, sig, p, g_out)
        torch.cuda.synchronize()
        fw, bw = [], []
        for _ in range(reps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            out = tape.forward(gbufs, cams, sig, p)
            e[1].record()
            g_out[:, 0] = 2 * (out[:, 0] - ref)
            tape.backward(gbufs, cams, sig, p, g_out)
            e[2].record()
            torch.cuda.synchronize()
            fw.append(e[0].elapsed_time(e[1]))
            bw.append(e[1].elapsed_time(e[2]))
        return statistics.median(fw), statistics.median(bw)

    # the stored schedule first, then the default (levels recomputed by the
    # backward), whose tape the fit below uses
    tape_s = dhrs.SvgfTape(W, H, frames, dhrs.TAPE_STORE)
    fwd_s, bwd_s = time_fb(tape_s)
    rec_bytes_s = tape_s.level_bytes(p.levels)
    tape_s.close()
    tape = dhrs.SvgfTape(W, H, frames, dhrs.TAPE_RECOMPUTE)
    fwd, bwd = time_fb(tape)
    # algorithmic bytes per pixel and frame (each buffer read or written once
    # per kernel): forward 340 as the SVGF frame + the records of a recorded
    # frame (weight sums 8 per level, last output 16); backward per level pass A 176 (input 16,
    # G-buffer 16, weight sums 8, output 16, upstream gradient 16, sigma
    # terms 32 read + written, records 64 written) and pass B 112 (records
    # 64, input 16, G-buffer 16, gradient 16 written), temporal backward 180;
    # recomputing the levels of every frame but the last two (whose records
    # the forward leaves in place): the forward's five levels (56 + 3 x 48 +
    # 40) + their records (5 x 8 + 16) = 296
    L = p.levels
    px = W * H
    bwd_px = L * (176 + 112) + 180
    # (the recomputing tape's forward records only the last two frames)
    bytes_fwd = frames * px * 340 + min(frames, 2) * px * (L * 8 + 16)
    bytes_bwd = frames * px * bwd_px + max(frames - 2, 0) * px * 296
    bytes_bwd_s = frames * px * bwd_px
    bytes_fb = bytes_fwd + bytes_bwd
    log_s = torch.tensor([0.0, 4.852, 1.386], device="cuda").requires_grad_(True)  # log(1, 128, 4)
    opt = torch.optim.Adam([log_s], lr=0.05)
    losses = []
    for _ in range(fit_steps):
        opt.zero_grad()
        o = dhrs.svgf_sequence(sig, log_s.exp(), gbufs, cams, p, tape)
        loss = ((o[:, 0] - ref) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(round(float(loss.detach()), 6))
    peak = _peaks()[0].get("hbm_gbs")
    gbs_b = bytes_bwd / (bwd * 1e-3) / 1e9
    gbs_bs = bytes_bwd_s / (bwd_s * 1e-3) / 1e9
    traffic = {k: _traffic(k) for k in ("atrous_bwd_a", "atrous_bwd_b", "temporal_bwd_kernel")}
    return {"workload": f"{frames} frames x {W}x{H}, terrain776k", "schedule": "levels recomputed",
            "forward_ms": round(fwd, 3), "backward_ms": round(bwd, 3),
            "level_record_bytes": tape.level_bytes(L),
            "algorithmic_gb_per_s": round(bytes_fb / ((fwd + bwd) * 1e-3) / 1e9, 1),
            "backward_algorithmic_gb_per_s": round(gbs_b, 1),
            "backward_frac_hbm": round(gbs_b / peak, 4) if peak else None,
            "backward_bytes_per_px_frame": bwd_px, "recompute_bytes_per_px_frame": 296,
            "stored_levels": {"forward_ms": round(fwd_s, 3), "backward_ms": round(bwd_s, 3),
                              "level_record_bytes": rec_bytes_s,
                              "backward_frac_hbm": round(gbs_bs / peak, 4) if peak else None},
            "ncu_dram_bytes_per_launch": traffic,
            "l2_vs_255spp_fit": losses, "sigmas_after_fit": [round(float(v), 4) for v in log_s.detach().exp()]}


def cpu_baseline(scene_d, cams, sample_px=4096, seed=7, rays_per_frame=None):
    """The oracle as it stands (brute force over all triangles, fp64, OpenMP
    on every host core) on a bounded sample of the same workload: primary,
    shadow and AO rays of `sample_px` seeded pixels of frame 0, and the
    full-frame SVGF at 1920x1080 (second frame, warm history) on the first
    two frames of the terrain camera spline over a coarse copy of the terrain
    scene (the same seeded heightfield on a 24 x 24 grid, 8 icospheres, 8
    boxes; 1,794 triangles), which the oracle traces in seconds (a
    brute-force trace of the 776k-triangle frame would take hours)."""
    import numpy as np

    import oracle as orc
    import workloads as wl
    S = orc.Scene(scene_d)
    r = np.random.default_rng(seed)
    pix = np.stack([r.integers(0, W, sample_px), r.integers(0, H, sample_px)], -1)
    t0 = time.perf_counter()
    tr = orc.trace(S, cams[0], orc.TraceParams(frame=0), pixels=pix)
    dt = time.perf_counter() - t0
    fg = int((tr["mesh"] != 0xFFFFFFFF).sum())
    n_rays = sample_px + 2 * fg
    coarse = wl.scene_terrain(n_spheres=8, n_boxes=8, sphere_level=1, terrain_n=24)
    B = orc.Scene(coarse)
    bc = wl.spline_path(coarse["terrain"], N_FRAMES, W, H)[:2]
    st = orc.SvgfState(W, H)
    svgf_s = 0.0
    for f, cam in enumerate(bc):
        t = orc.trace(B, cam, orc.TraceParams(frame=f))
        zn, mesh = orc.gbuffer_f32(t, W, H)
        t1 = time.perf_counter()
        st.frame(zn, mesh, cam, t["shadow_mask"].reshape(H, W), t["ao_count"].reshape(H, W), orc.SvgfParams())
        svgf_s = time.perf_counter() - t1
    return {"value": round(n_rays / dt / 1e6, 6), "unit": "Mrays/s", "cores": orc.num_threads(),
            "kind": "oracle", "ns_per_ray": round(dt / n_rays * 1e9, 1),
            "svgf_ms_per_frame_1080p": round(svgf_s * 1e3, 1),
            "trace_s_per_frame_extrapolated": (round(dt / n_rays * rays_per_frame, 1) if rays_per_frame else None),
            "sample": f"{sample_px} seeded pixels of frame 0 (primary + shadow + AO rays, "
                      f"{n_rays} rays, {dt:.1f} s) of the 1920x1080 776,050-triangle workload; "
                      f"SVGF: one full 1920x1080 frame with history (terrain spline frame 1 over the "
                      f"1,794-triangle coarse terrain, traced by the oracle)"}


def run_denoise_variants(sc, scene_d, frames=12, W=1280, H=720, levels=(0, 1, 2, 5, (1, 3), (2, 3))):
    """Lightweight denoiser variants: the same noisy 1-spp frames filtered
    with 0, 1, 2 and 5 a-trous levels of the 5x5 kernel, and 1 and 2 levels
    of the smaller 3x3 kernel; error of the filtered AO of the last 4 frames
    against a 255-spp AO reference, and SVGF time per frame."""
    import numpy as np
    import torch

    import paper_2406_06963_b300 as dhrs
    import workloads as wl
    cams = wl.spline_path(scene_d["terrain"], N_FRAMES, W, H)[:frames]
    gbufs, masks, aos, refs = [], [], [], []
    for f, cam in enumerate(cams):
        g = dhrs.GBuffer(W, H)
        m = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        a = torch.empty_like(m)
        dhrs.trace_visibility(sc, cam, dhrs.TraceParams(ao_spp=1, frame=f), g, m, a)
        g2 = dhrs.GBuffer(W, H)
        a2 = torch.empty_like(m)
        dhrs.trace_visibility(sc, cam, dhrs.TraceParams(ao_spp=255, frame=f), g2, m.clone(), a2)
        gbufs.append(g)
        masks.append(m)
        aos.append(a)
        refs.append(a2.float() / 255.0)
    out = {}
    ao = torch.empty((H, W), device="cuda")
    sh = torch.empty_like(ao)
    for L in levels:
        L, width = (L, 5) if isinstance(L, int) else L
        p = dhrs.SvgfParams(ao_spp=1, levels=L, kernel_width=width)
        st = dhrs.SvgfState(W, H)
        errs, ms = [], []
        for f, cam in enumerate(cams):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st.reconstruct(gbufs[f], gbufs[f - 1] if f else None, cam, cams[f - 1] if f else None, masks[f],
                           aos[f], p, ao, sh)
            e1.record()
            torch.cuda.synchronize()
            if f >= frames - 4:
                fg = torch.isfinite(gbufs[f].depth_normal[..., 0])
                d = (ao - refs[f])[fg]
                errs.append((float((d * d).mean()), float(d.abs().mean())))
                ms.append(e0.elapsed_time(e1))
        out[f"levels_{L}" + ("" if width == 5 else "_kernel_3x3")] = {"ao_rmse": round(float(np.sqrt(np.mean([e[0] for e in errs]))), 5),
                              "ao_mean_abs": round(float(np.mean([e[1] for e in errs])), 5),
                              "svgf_ms": round(float(np.median(ms)), 4)}
    noisy = [float(((aos[f].float() - refs[f])[torch.isfinite(gbufs[f].depth_normal[..., 0])] ** 2).mean())
             for f in range(frames - 4, frames)]
    out["noisy_1spp_ao_rmse"] = round(float(np.sqrt(np.mean(noisy))), 5)
    out["workload"] = f"{frames} frames x {W}x{H}, terrain776k, 1 spp, reference 255 spp, last 4 frames"
    return out


def run_selective(sc, scene_d, frames=30, resolution=4096):
    """Selective shadow rays (Section 5): the 1080p trace with shadow rays
    only where a 4096^2 shadow map cannot decide, against the full trace.
    Trace-only device time per frame (median, L2 flushed before each
    frame), share of foreground pixels whose shadow ray is called, and share
    whose shadow bit differs from the full trace's ray."""
    import numpy as np
    import torch

    import paper_2406_06963_b300 as dhrs
    import workloads as wl
    cams = wl.spline_path(scene_d["terrain"], N_FRAMES, W, H)
    light = dhrs.TraceParams().light_dirs[0]
    sm = dhrs.ShadowMap(sc, light, resolution)
    g = dhrs.GBuffer(W, H)
    mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
    ao = torch.empty_like(mask)
    rm = torch.empty_like(mask)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")

    def timed(fn):
        ts = []
        for f in range(frames):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn(f)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts[3:]))

    full_ms = timed(lambda f: dhrs.trace_visibility(sc, cams[f % N_FRAMES], dhrs.TraceParams(frame=f), g, mask, ao))
    sel_ms = timed(lambda f: dhrs.trace_visibility_selective(sc, cams[f % N_FRAMES], dhrs.TraceParams(frame=f),
                                                             [sm], g, mask, ao, rm))
    n_fg = n_called = n_diff = 0
    for f in (0, 15, 30, 45):
        p = dhrs.TraceParams(frame=f)
        dhrs.trace_visibility(sc, cams[f], p, g, mask, ao)
        full = mask.clone()
        dhrs.trace_visibility_selective(sc, cams[f], p, [sm], g, mask, ao, rm)
        fg = g.mesh.view(torch.int32) != -1
        called = (rm & 1) == 1
        n_fg += int(fg.sum())
        n_called += int((called & fg).sum())
        n_diff += int((fg & (full != mask)).sum())
    info = sm.info()
    return {"map_resolution": resolution, "map_build_ms": round(info["build_ms"], 3),
            "map_mb": round(info["bytes"] / 2**20, 1),
            "trace_ms_full": round(full_ms, 4), "trace_ms_selective": round(sel_ms, 4),
            "shadow_rays_called_frac": round(n_called / n_fg, 5),
            "shadow_bits_differing_frac": n_diff / n_fg,
            "workload": f"terrain776k 1920x1080, {frames} spline frames, 1 light, 0.5 deg cone"}


def run_reference(args):
    """Reference arm: the CPU oracle timed per step on a bounded pixel sample
    (the same metric and workload as ours)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    import numpy as np

    import oracle as orc
    import workloads as wl
    scene_d = wl.scene_terrain()
    cams = wl.spline_path(scene_d["terrain"], N_FRAMES, W, H)
    S = orc.Scene(scene_d)
    r = np.random.default_rng(11)
    per_step = args.ref_pixels

    def step(i):
        pix = np.stack([r.integers(0, W, per_step), r.integers(0, H, per_step)], -1)
        tr = orc.trace(S, cams[i % N_FRAMES], orc.TraceParams(frame=i), pixels=pix)
        return per_step + 2 * int((tr["mesh"] != 0xFFFFFFFF).sum())

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    n = sum(step(args.warmup + i) for i in range(args.steps))
    dt = time.perf_counter() - t0
    v = n / dt / 1e6
    sample = f"{per_step} seeded pixels per step (primary + shadow + AO rays) of the 1920x1080 " \
             f"776,050-triangle workload"
    return {"metric": METRIC, "value": round(v, 6), "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(ws, len(scene_d["indices"])),
            "impl": "reference",
            "cpu_baseline": {"value": round(v, 6), "unit": "Mrays/s", "cores": orc.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 6), "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the serving, FP16 and adjoint measurements")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-pixels", type=int, default=4096)
    ap.add_argument("--ref-pixels", type=int, default=24)
    ap.add_argument("--primary", default="raster", choices=["raster", "traverse"],
                    help="primary visibility of the session frames: the rasteriser (default) or BVH "
                         "traversal (same outputs)")
    ap.add_argument("--selective-only", action="store_true",
                    help="print only the selective shadow ray measurement (profiling aid)")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="print only the adjoint measurement (profiling aid)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.selective_only:
        import paper_2406_06963_b300 as dhrs
        import workloads as wl
        scene_d = wl.scene_terrain()
        print(json.dumps({"selective_shadows": run_selective(dhrs.Scene(scene_d), scene_d,
                                                             frames=args.steps + args.warmup)}), flush=True)
        return
    if args.adjoint_only:
        import paper_2406_06963_b300 as dhrs
        import workloads as wl
        scene_d = wl.scene_terrain()
        print(json.dumps({"adjoint": run_adjoint(dhrs.Scene(scene_d), scene_d)}), flush=True)
        return
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
