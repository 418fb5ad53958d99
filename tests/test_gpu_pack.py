"""Lossless packing of the raw trace outputs (dhr_visibility_pack): a plain
decoder written from the stream format in dhrs.h reproduces the bitmask
and AO count bit for bit, on traced frames, ragged sizes, several lights
and AO sample counts, and on uniform and random inputs."""
import numpy as np
import pytest

import paper_2406_06963_b300 as dhrs
import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def decode(words: np.ndarray):
    """The stream format of dhrs.h, decoded pixel by pixel."""
    w = words.astype(np.uint32)
    assert w[0] == 0x56524844
    W, H = int(w[1]), int(w[2])
    n_lights, ao_bits = int(w[3] & 0xFF), int((w[3] >> 8) & 0xFF)
    M = int(w[4])
    planes = n_lights + ao_bits
    tx, ty = (W + 31) // 32, (H + 7) // 8
    T = tx * ty
    n_class = (planes * T + 15) // 16
    assert len(w) == 5 + n_class + 8 * M
    mask = np.zeros((H, W), np.uint8)
    ao = np.zeros((H, W), np.uint8)
    m = 0
    for pl in range(planes):
        plane = np.zeros((ty * 8, tx * 32), np.uint8)
        for t in range(T):
            k = pl * T + t
            c = (int(w[5 + k // 16]) >> (2 * (k % 16))) & 3
            y0, x0 = (t // tx) * 8, (t % tx) * 32
            if c == 1:
                plane[y0:y0 + 8, x0:x0 + 32] = 1
            elif c == 2:
                rows = w[5 + n_class + 8 * m: 5 + n_class + 8 * m + 8]
                bits = (rows[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1
                plane[y0:y0 + 8, x0:x0 + 32] = bits.astype(np.uint8)
                m += 1
            else:
                assert c == 0
        plane = plane[:H, :W]
        if pl < n_lights:
            mask |= plane << pl
        else:
            ao |= plane << (pl - n_lights)
    assert m == M
    return mask, ao


def _check(mask, ao, n_lights, spp):
    H, W = mask.shape
    words = dhrs.pack_visibility(mask, ao, n_lights, spp)
    torch.cuda.synchronize()
    dm, da = decode(words.cpu().numpy().view(np.uint32))
    assert np.array_equal(dm, mask.cpu().numpy()) and np.array_equal(da, ao.cpu().numpy())
    assert words.numel() * 4 <= dhrs.lib().dhr_visibility_pack_bound(W, H, n_lights, spp)
    return words.numel() * 4


@pytest.mark.parametrize("w,h,lights,spp", [(256, 256, 1, 1), (37, 23, 3, 8), (300, 7, 2, 255), (1, 1, 1, 1)])
def test_pack_round_trip_on_traced_frames(w, h, lights, spp):
    s = wl.scene_boxes()
    sc = dhrs.Scene(s)
    cam = wl.boxes_camera(w, h)
    dirs = [(0.3, 1.0, 0.2), (-0.6, 0.8, 0.3), (0.2, 0.5, -0.8)][:lights]
    tp = dhrs.TraceParams(light_dirs=dirs, cone_half_angle_deg=[0.5, 3.0, 1.5][:lights], ao_spp=spp, frame=3)
    g = dhrs.GBuffer(w, h)
    mask = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    ao = torch.empty_like(mask)
    dhrs.trace_visibility(sc, cam, tp, g, mask, ao)
    _check(mask, ao, lights, spp)


def test_pack_uniform_and_random_inputs():
    H, W = 120, 200
    zero = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
    ones = torch.ones_like(zero)
    size0 = _check(zero, zero, 1, 1)
    assert size0 == 4 * (5 + (2 * 7 * 15 + 15) // 16)       # every tile uniform: no tile words
    assert _check(ones, ones, 1, 1) == size0
    g = torch.Generator(device="cuda").manual_seed(5)
    rm = torch.randint(0, 8, (H, W), dtype=torch.uint8, device="cuda", generator=g)
    ra = torch.randint(0, 9, (H, W), dtype=torch.uint8, device="cuda", generator=g)
    _check(rm, ra, 3, 8)


def test_pack_rejects_bad_parameters():
    assert dhrs.lib().dhr_visibility_pack_bound(0, 10, 1, 1) == 0
    assert dhrs.lib().dhr_visibility_pack_bound(10, 10, 9, 1) == 0
    assert dhrs.lib().dhr_visibility_pack_bound(10, 10, 1, 256) == 0
    m = torch.zeros((10, 10), dtype=torch.uint8, device="cuda")
    with pytest.raises(dhrs.DhrError):
        dhrs.pack_visibility(m, m, 0, 1)
