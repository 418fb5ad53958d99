"""The largest session the library accepts, 16384 x 16384 (2^28 pixels,
where pixel indices still fit the kernels' 32-bit arithmetic): two frames
through dhr_step_frame, the trace of sampled pixels (corners and the very
last pixel included) against the oracle, and the filtered planes finite,
within [0, 1] and exactly 1 on background pixels."""
import numpy as np
import pytest

import oracle as orc
import paper_2406_06963_b300 as dhrs
import workloads as wl
from gpu_util import compare_trace

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


def _view(ptr, shape, typestr):
    return torch.as_tensor(dhrs._DevArray(ptr, shape, typestr), device="cuda")


def test_maximum_session_size():
    W = H = 16384
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    cams = wl.orbit_path(2, W, H, degrees=2.0)
    sess = dhrs.Session(sc, W, H, trace=dhrs.TraceParams(ao_spp=2), svgf=dhrs.SvgfParams(ao_spp=2))
    ao = torch.empty((H, W), device="cuda")
    sh = torch.empty_like(ao)
    for f, cam in enumerate(cams):
        sess.step(cam, f, ao, sh)
    torch.cuda.synchronize()
    n = W * H
    fb = sess.frame_buffers()
    zn = _view(fb["depth_normal"], (n, 4), "<f4")
    mesh = _view(fb["mesh"], (n,), "<i4")
    mask = _view(fb["mask"], (n,), "|u1")
    aoc = _view(fb["ao"], (n,), "|u1")
    r = np.random.default_rng(9)
    pix = np.concatenate([np.stack([r.integers(0, W, 256), r.integers(0, H, 256)], -1),
                          [[W - 1, H - 1], [0, H - 1], [W - 1, 0], [0, 0]]]).astype(np.int64)
    idx = torch.from_numpy(pix[:, 1] * W + pix[:, 0]).cuda()
    z = zn[idx].cpu().numpy().astype(np.float64)
    gpu = dict(depth=z[:, 0], normal=z[:, 1:], mesh=mesh[idx].cpu().numpy().view(np.uint32),
               shadow_mask=mask[idx].cpu().numpy(), ao_count=aoc[idx].cpu().numpy())
    ref = orc.trace(orc.Scene(s), cams[-1], orc.TraceParams(ao_spp=2, frame=1), pixels=pix)
    res = compare_trace(gpu, ref, np.arange(len(pix)), 1, 2)
    assert res["primary_unexplained"] == 0 and res["shadow_unexplained"] == 0 and res["ao_unexplained"] == 0, res
    assert res["depth_rel_max"] < 2e-5 and res["normal_abs_max"] < 2e-5, res
    bg = mesh == -1                       # 0xFFFFFFFF: no hit
    assert bool(bg.any()) and not bool(bg.all())
    for out in (ao, sh):
        v = out.view(-1)
        assert bool(torch.isfinite(v).all())
        assert float(v.min()) >= -1e-6 and float(v.max()) <= 1 + 1e-6
        assert bool((v[bg] == 1.0).all())
