"""Pins for the oracle's random numbers and ray-direction sampling.

Section 3.1 (cone-jittered shadow rays) and Section 3.2 (cosine-weighted AO
rays).  The generator is pcg4d (Jarzynski & Olano 2020); it is pinned by its
inverse (undoing each published step in reverse order), by exact values of
the 24-bit mapping, and by the closed-form moments of the distributions
the directions must follow.
"""
import math

import numpy as np
import pytest
from scipy import stats

M32 = 0xFFFFFFFF


def _pcg4d_inverse(v):
    """Undo pcg4d step by step (Python integers)."""
    x, y, z, w = [int(a) for a in v]
    # second mixing, reversed
    w = (w - y * z) & M32
    z = (z - x * y) & M32
    y = (y - z * x) & M32
    x = (x - y * w) & M32
    # x ^= x >> 16 is its own inverse on 32 bits
    x, y, z, w = [a ^ (a >> 16) for a in (x, y, z, w)]
    # first mixing, reversed
    w = (w - y * z) & M32
    z = (z - x * y) & M32
    y = (y - z * x) & M32
    x = (x - y * w) & M32
    inv = pow(1664525, -1, 1 << 32)
    return [((a - 1013904223) * inv) & M32 for a in (x, y, z, w)]


def test_pcg4d_inverts(orc):
    r = np.random.default_rng(1)
    for _ in range(2000):
        v = r.integers(0, 1 << 32, 4, dtype=np.uint64).astype(np.uint32)
        h = orc.pcg4d(v)
        assert _pcg4d_inverse(h) == [int(a) for a in v]


def test_pcg4d_avalanche(orc):
    """One flipped bit in the low 16 bits of an input lane (where pixel
    coordinates, frame and sample counters live) changes about half of the
    24 output bits that become uniforms."""
    r = np.random.default_rng(2)
    flips = []
    for _ in range(1000):
        v = r.integers(0, 1 << 32, 4, dtype=np.uint64).astype(np.uint32)
        lane, bit = r.integers(0, 4), r.integers(0, 16)
        v2 = v.copy()
        v2[lane] ^= np.uint32(1 << int(bit))
        a, b = orc.pcg4d(v), orc.pcg4d(v2)
        flips.append(sum(bin((int(x) ^ int(y)) >> 8).count("1") for x, y in zip(a, b)) / 96.0)
    assert abs(np.mean(flips) - 0.5) < 0.02


def test_u24_exact(orc):
    assert orc.u24(0) == 0.0
    assert orc.u24(255) == 0.0
    assert orc.u24(256) == 2.0 ** -24
    assert orc.u24(0xFFFFFFFF) == (2 ** 24 - 1) / 2 ** 24
    assert orc.u24(0x80000000) == 0.5


def _disk_samples(orc, n, ray_type=1, frame=3):
    pts = np.array([orc.disk_point(i % 97, i // 97, frame, 0, ray_type, 0) for i in range(n)])
    return pts[:, 0], pts[:, 1], pts[:, 2].astype(int)


def test_disk_uniform(orc):
    """Uniform on the unit disk: r^2 ~ U[0,1), angle ~ U[0, 2pi)."""
    x, y, k = _disk_samples(orc, 20000)
    r2 = x * x + y * y
    assert r2.max() < 1.0
    assert stats.kstest(r2, "uniform").pvalue > 1e-3
    ang = (np.arctan2(y, x) + 2 * np.pi) % (2 * np.pi) / (2 * np.pi)
    assert stats.kstest(ang, "uniform").pvalue > 1e-3
    # accepted candidate index is geometric with success probability pi/4
    p = math.pi / 4
    counts = np.bincount(k, minlength=9)[:4]
    expect = np.array([p * (1 - p) ** j for j in range(4)]) * len(k)
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < stats.chi2.ppf(0.9999, 3)


def test_u24_uniform_chi2(orc):
    """The 24-bit uniforms of neighbouring pixels are uniform and uncorrelated."""
    us = []
    for px in range(4096):
        h = orc.pcg4d([px, 7, 11, 1 << 24])
        us.append([orc.u24(int(a)) for a in h])
    us = np.array(us)
    for lane in range(4):
        c, _ = np.histogram(us[:, lane], bins=32, range=(0, 1))
        assert stats.chisquare(c).pvalue > 1e-4
    assert abs(np.corrcoef(us[:-1, 0], us[1:, 0])[0, 1]) < 0.06
    assert abs(np.corrcoef(us[:, 0], us[:, 1])[0, 1]) < 0.06


NORMALS = [(0, 0, 1), (0, 0, -1), (0, 1, 0), (1, 0, 0), (0.6, 0.0, -0.8),
           (0.48, 0.6, 0.64), (-0.36, -0.48, 0.8)]


@pytest.mark.parametrize("n", NORMALS)
def test_onb_orthonormal(orc, n):
    n = np.array(n, np.float32)
    T, B = orc.onb_f32(n)
    T, B, nn = T.astype(float), B.astype(float), n.astype(float)
    for a in (T, B):
        assert abs(np.dot(a, a) - 1) < 1e-6
        assert abs(np.dot(a, nn)) < 1e-6
    assert abs(np.dot(T, B)) < 1e-6
    assert np.allclose(np.cross(T, B), nn, atol=1e-6)      # right-handed: T x B = n


@pytest.mark.parametrize("n", NORMALS)
def test_ao_cosine_weighted(orc, n):
    """Section 3.2: cosine-weighted hemisphere.  E[cos] = 2/3, E[cos^2] = 1/2,
    zero mean tangential components, unit length, never below the surface."""
    n = np.array(n, np.float32)
    N = 6000
    normals = np.tile(n, (N, 1))
    px = np.arange(N) % 101
    py = np.arange(N) // 101
    out = orc.sample_batch(px, py, 5, 0, 0, normals, [0, 1, 0], 0.0)
    d = out["dir_ao"].astype(np.float64)
    c = d @ n.astype(np.float64)
    assert np.all(np.abs((d * d).sum(1) - 1) < 1e-6)
    assert c.min() >= -1e-7
    se = 1.0 / math.sqrt(N)
    assert abs(c.mean() - 2 / 3) < 4 * math.sqrt(1 / 2 - 4 / 9) * se
    assert abs((c * c).mean() - 0.5) < 4 * math.sqrt(1 / 3 - 1 / 4) * se
    T, B = orc.onb_f32(n)
    assert abs((d @ T.astype(float)).mean()) < 0.04
    assert abs((d @ B.astype(float)).mean()) < 0.04
    # P(cos <= c) = c^2 under a cosine-weighted pdf
    assert stats.kstest(c * c, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("deg", [0.5, 5.0, 20.0])
def test_cone_bounded_uniform(orc, deg):
    """Section 3.1: shadow ray offset inside the light's cone, unit length.
    Tangent-disk form: tan(angle to l) / tan(theta) is the radius of a
    uniform disk point, so its square is U[0,1)."""
    l = np.array([0.3, 1.0, 0.2])
    l = (l / np.linalg.norm(l)).astype(np.float32)
    t = orc.tan_f32(math.radians(deg))
    N = 6000
    px = np.arange(N) % 89
    py = np.arange(N) // 89
    out = orc.sample_batch(px, py, 9, 0, 0, np.tile([0, 0, 1], (N, 1)), l, t)
    d = out["dir_sh"].astype(np.float64)
    assert np.all(np.abs((d * d).sum(1) - 1) < 1e-6)
    cosang = np.clip(d @ l.astype(np.float64), -1, 1)
    ang = np.arccos(cosang)
    assert ang.max() <= math.radians(deg) * (1 + 1e-4) + 1e-6
    rho = np.tan(ang) / math.tan(math.radians(deg))
    assert stats.kstest(rho * rho, "uniform").pvalue > 1e-3


def test_cone_zero_is_light_direction(orc):
    """A zero cone angle reproduces the hard-shadow ray toward the light centre
    (Section 2.2 / Fig. 1a)."""
    l = np.array([0.3, 1.0, 0.2])
    l = (l / np.linalg.norm(l)).astype(np.float32)
    for i in range(50):
        x, y, _ = orc.disk_point(i, 3, 0, 0, 0, 0)
        d = orc.cone_dir_f32(l, 0.0, x, y)
        assert np.allclose(d, l, atol=1.5e-7)
