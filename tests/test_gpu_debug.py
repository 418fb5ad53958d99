"""The bounds-checked debug build (libdhrs_debug.so, DHR_DEBUG) on small cases.

Every path runs on ragged image sizes (tiles cut by the image border) in a
child process that loads libdhrs_debug.so (DHRS_DEBUG=1): tracing with
traversed and rasterised primaries, selective shadow rays, the SVGF in both
storage forms and both kernel widths, the pipelined session, the adjoint,
the batched server (with warp targets, traced and rasterised) and the
packer.  No gather index may leave its buffer
(dhr_debug_status reports no event).  The self test then makes one checked
out-of-range read, which must be reported with its site and index; the
check redirects the read, so nothing outside a buffer is touched.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json
import numpy as np
import torch
import paper_2406_06963_b300 as dhrs
import workloads as wl

res = {}
err, dbg = dhrs.debug_status()
res["debug_build"] = dbg
sc = dhrs.Scene(wl.scene_boxes())
W, H = 203, 77
cams = wl.orbit_path(4, W, H, degrees=6.0)
mask = torch.empty((H, W), dtype=torch.uint8, device="cuda")
ao = torch.empty_like(mask)
for prim in (dhrs.PRIMARY_TRAVERSE, dhrs.PRIMARY_RASTER):
    for prec in (dhrs.DHR_FP32, dhrs.DHR_FP16):
        g = dhrs.GBuffer(W, H, prec)
        tp = dhrs.TraceParams(light_dirs=[(0.3, 1.0, 0.2), (-0.5, 0.8, 0.1)], cone_half_angle_deg=[0.5, 2.0],
                              ao_spp=2, primary=prim)
        dhrs.trace_visibility(sc, cams[0], tp, g, mask, ao)
sm = dhrs.ShadowMap(sc, (0.3, 1.0, 0.2), resolution=256)
g = dhrs.GBuffer(W, H)
dhrs.trace_visibility_selective(sc, cams[1], dhrs.TraceParams(ao_spp=1), [sm], g, mask, ao)
res["trace"] = dhrs.debug_status()[0]

o1 = torch.empty((H, W), device="cuda")
o2 = torch.empty_like(o1)
for prec in (dhrs.DHR_FP32, dhrs.DHR_FP16):
    for kw, levels in ((5, 5), (3, 1), (5, 0)):
        st = dhrs.SvgfState(W, H, prec)
        gs = [dhrs.GBuffer(W, H, prec) for _ in cams]
        for f, cam in enumerate(cams):
            dhrs.trace_visibility(sc, cam, dhrs.TraceParams(ao_spp=1, frame=f), gs[f], mask, ao)
            st.reconstruct(gs[f], gs[f - 1] if f else None, cam, cams[f - 1] if f else None, mask, ao,
                           dhrs.SvgfParams(ao_spp=1, levels=levels, kernel_width=kw), o1, o2)
res["svgf"] = dhrs.debug_status()[0]

sess = dhrs.Session(sc, W, H)
for f, cam in enumerate(cams):
    sess.step(cam, f, o1, o2)
res["session"] = dhrs.debug_status()[0]

F = 3
gbs = []
for f in range(F):
    gg = dhrs.GBuffer(W, H)
    dhrs.trace_visibility(sc, cams[f], dhrs.TraceParams(ao_spp=1, frame=f), gg, mask, ao)
    gbs.append(gg)
r = np.random.default_rng(0)
sig = torch.from_numpy(r.uniform(0.05, 0.95, (F, 2, H, W)).astype(np.float32)).cuda()
gout = torch.from_numpy(r.normal(size=(F, 2, H, W)).astype(np.float32)).cuda()
for sched in (dhrs.TAPE_RECOMPUTE, dhrs.TAPE_STORE):
    tape = dhrs.SvgfTape(W, H, F, sched)
    for levels in (5, 2, 1, 0):
        p = dhrs.SvgfParams(levels=levels)
        tape.forward(gbs, cams[:F], sig, p)
        tape.backward(gbs, cams[:F], sig, p, gout)
        tape.backward(gbs, cams[:F], sig, p, gout)
res["adjoint"] = dhrs.debug_status()[0]

paths = [cams, wl.orbit_path(4, 96, 50, degrees=9.0, start_deg=40)]
for raster_min in (None, 0):   # primary rays; every session and warp target rasterised
    srv = dhrs.Server(sc, 4 << 30)
    if raster_min is not None:
        srv.set_raster_min_pixels(raster_min)
    ids = [srv.open(W, H), srv.open(96, 50)]
    for f in range(3):
        for k, sid in enumerate(ids):
            srv.submit(sid, paths[k][f], f, dhrs.now_ns(), 10 * k + f, cam_target=paths[k][f + 1])
        srv.pump()
        done = srv.poll(wait=True)
        while len([d for d in done if not d["dropped"]]) < len(ids):
            done += srv.poll(wait=True)
    srv.close()
res["server"] = dhrs.debug_status()[0]

dhrs.pack_visibility(mask, ao, 1, 1)
res["pack"] = dhrs.debug_status()[0]

dhrs.debug_selftest()
res["selftest"] = dhrs.debug_status()[0]
res["after_selftest"] = dhrs.debug_status()[0]
print("RESULT " + json.dumps(res))
'''


def test_debug_build_checks_every_gather():
    from paper_2406_06963_b300 import build
    build.build(debug=True)
    env = dict(os.environ, DHRS_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    print(res)
    assert res["debug_build"] is True
    for path in ("trace", "svgf", "session", "adjoint", "server", "pack"):
        assert res[path] == 0, (path, hex(res[path]))
    # the self test's event: flag, site 11, index 5; reading clears it
    ev = res["selftest"]
    assert ev >> 63 == 1 and (ev >> 40) & 0xFF == 11 and ev & 0xFFFFFFFFFF == 5, hex(ev)
    assert res["after_selftest"] == 0
