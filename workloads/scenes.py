"""Seeded synthetic scenes standing in for the paper's test scenes.

The paper evaluates on PINK ROOM, SUN TEMPLE and BISTRO (Section 4.1), none of
which is available here.  These generators build triangle soups of the same
kind (a ground, many closed objects resting on it) from numpy PCG64 streams.
They hold geometry construction only; no ray tracing or filtering arithmetic
lives here, so both the CUDA path and the CPU oracle may consume them.

Every scene is returned as a dict:
    vertices  float32 [n_vertices, 3]
    indices   uint32  [n_triangles, 3]   (counter-clockwise seen from outside)
    mesh_ids  uint32  [n_triangles]      (one id per object; 0 = ground)
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2406_06963


def rng_for(index: int) -> np.random.Generator:
    """numpy PCG64 stream for workload ``index`` (seed = 240606963 + index)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


# --------------------------------------------------------------------------
# primitive meshes
# --------------------------------------------------------------------------
def box_mesh(lo, hi):
    """Axis-aligned box with outward-facing counter-clockwise triangles."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    c = np.array([[lo[0] if (i & 1) == 0 else hi[0],
                   lo[1] if (i & 2) == 0 else hi[1],
                   lo[2] if (i & 4) == 0 else hi[2]] for i in range(8)])
    # faces as quads (a, b, c, d) counter-clockwise seen from outside
    quads = [(0, 4, 6, 2),   # -x
             (1, 3, 7, 5),   # +x
             (0, 1, 5, 4),   # -y
             (2, 6, 7, 3),   # +y
             (0, 2, 3, 1),   # -z
             (4, 5, 7, 6)]   # +z
    tris = []
    for a, b, cc, d in quads:
        tris.append((a, b, cc))
        tris.append((a, cc, d))
    return c, np.array(tris, np.int64)


def icosphere(level: int):
    """Unit icosphere: the regular icosahedron subdivided ``level`` times."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, np.int64)


class _Builder:
    def __init__(self):
        self.v, self.i, self.m = [], [], []
        self.nv = 0

    def add(self, verts, tris, mesh_id):
        self.v.append(np.asarray(verts, np.float64))
        self.i.append(np.asarray(tris, np.int64) + self.nv)
        self.m.append(np.full(len(tris), mesh_id, np.int64))
        self.nv += len(verts)

    def done(self, **extra):
        out = dict(vertices=np.concatenate(self.v).astype(np.float32),
                   indices=np.concatenate(self.i).astype(np.uint32),
                   mesh_ids=np.concatenate(self.m).astype(np.uint32))
        out.update(extra)
        return out


# --------------------------------------------------------------------------
# 256x256 scene: ground plane + 16 boxes (194 triangles)
# --------------------------------------------------------------------------
def scene_boxes(index: int = 0, n_boxes: int = 16):
    """Ground quad [-10,10]^2 at y=0 plus ``n_boxes`` boxes resting on it.

    Box edge lengths are U[0.2, 1.5] per axis, box centres U[-5, 5]^2.
    """
    r = rng_for(index)
    b = _Builder()
    g = np.array([[-10, 0, -10], [10, 0, -10], [10, 0, 10], [-10, 0, 10]], np.float64)
    b.add(g, [(0, 3, 2), (0, 2, 1)], 0)           # normal +y
    for k in range(n_boxes):
        e = r.uniform(0.2, 1.5, 3)
        c = r.uniform(-5.0, 5.0, 2)
        lo = np.array([c[0] - e[0] / 2, 0.0, c[1] - e[2] / 2])
        hi = np.array([c[0] + e[0] / 2, e[1], c[1] + e[2] / 2])
        v, t = box_mesh(lo, hi)
        b.add(v, t, k + 1)
    return b.done(name="boxes194")


# --------------------------------------------------------------------------
# ~776k-triangle scene: heightfield terrain + 2000 icospheres + 500 boxes
# --------------------------------------------------------------------------
def _value_noise(r: np.random.Generator, xs, zs, cells: int, extent: float):
    """Smooth value noise in [-1, 1]: random lattice values, smoothstep blend."""
    lat = r.uniform(-1.0, 1.0, (cells + 2, cells + 2))
    fx = (xs + extent) / (2 * extent) * cells
    fz = (zs + extent) / (2 * extent) * cells
    ix = np.clip(np.floor(fx).astype(np.int64), 0, cells)
    iz = np.clip(np.floor(fz).astype(np.int64), 0, cells)
    tx = fx - ix
    tz = fz - iz
    sx = tx * tx * (3 - 2 * tx)
    sz = tz * tz * (3 - 2 * tz)
    a = lat[iz, ix] * (1 - sx) + lat[iz, ix + 1] * sx
    c = lat[iz + 1, ix] * (1 - sx) + lat[iz + 1, ix + 1] * sx
    return a * (1 - sz) + c * sz


class Terrain:
    """256x256-vertex heightfield over [-128, 128]^2, amplitude 8."""

    def __init__(self, r: np.random.Generator, n: int = 256, extent: float = 128.0):
        self.n, self.extent = n, extent
        xs = np.linspace(-extent, extent, n)
        X, Z = np.meshgrid(xs, xs)          # X varies along columns
        h = 0.75 * _value_noise(r, X, Z, 8, extent) + 0.25 * _value_noise(r, X, Z, 32, extent)
        self.heights = 8.0 * h              # [n_z, n_x]
        self.xs = xs

    def height_at(self, x, z):
        """Bilinear interpolation of the vertex grid (the mesh surface)."""
        n, e = self.n, self.extent
        fx = np.clip((x + e) / (2 * e) * (n - 1), 0, n - 1 - 1e-9)
        fz = np.clip((z + e) / (2 * e) * (n - 1), 0, n - 1 - 1e-9)
        ix, iz = int(fx), int(fz)
        tx, tz = fx - ix, fz - iz
        H = self.heights
        a = H[iz, ix] * (1 - tx) + H[iz, ix + 1] * tx
        c = H[iz + 1, ix] * (1 - tx) + H[iz + 1, ix + 1] * tx
        return float(a * (1 - tz) + c * tz)

    def mesh(self):
        n = self.n
        X, Z = np.meshgrid(self.xs, self.xs)
        verts = np.stack([X, self.heights, Z], -1).reshape(-1, 3)
        iz, ix = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
        a = (iz * n + ix).ravel()
        b = a + 1
        c = a + n
        d = c + 1
        # normals +y: (a, c, b) and (b, c, d) are counter-clockwise from above
        t1 = np.stack([a, c, b], -1)
        t2 = np.stack([b, c, d], -1)
        return verts, np.concatenate([t1, t2])


def scene_terrain(index: int = 1, n_spheres: int = 2000, n_boxes: int = 500,
                  sphere_level: int = 2, terrain_n: int = 256):
    """Terrain + icospheres (r in U[0.1, 2]) + boxes (edges U[0.2, 4]).

    All objects rest on the terrain; at the default sizes this is 776,050
    triangles in one flattened soup (mesh id 0 = terrain, 1..n_spheres =
    spheres, then boxes).
    """
    r = rng_for(index)
    terr = Terrain(r, n=terrain_n)
    b = _Builder()
    tv, tt = terr.mesh()
    b.add(tv, tt, 0)
    sv, st = icosphere(sphere_level)
    lim = terr.extent - 8.0
    for k in range(n_spheres):
        rad = r.uniform(0.1, 2.0)
        x, z = r.uniform(-lim, lim, 2)
        y = terr.height_at(x, z) + rad
        b.add(sv * rad + np.array([x, y, z]), st, 1 + k)
    for k in range(n_boxes):
        e = r.uniform(0.2, 4.0, 3)
        x, z = r.uniform(-lim, lim, 2)
        y0 = terr.height_at(x, z)
        v, t = box_mesh([x - e[0] / 2, y0, z - e[2] / 2], [x + e[0] / 2, y0 + e[1], z + e[2] / 2])
        b.add(v, t, 1 + n_spheres + k)
    out = b.done(name="terrain776k")
    out["terrain"] = terr
    return out


def scene_enclosing_sphere(radius: float = 0.4, level: int = 3):
    """A closed icosphere (used with a camera placed at its centre)."""
    v, t = icosphere(level)
    b = _Builder()
    b.add(v * radius, t, 0)
    return b.done(name="sphere")


def scene_quad(corners, mesh_id: int = 0):
    """One planar quad given by four corners (counter-clockwise)."""
    b = _Builder()
    b.add(np.asarray(corners, np.float64), [(0, 1, 2), (0, 2, 3)], mesh_id)
    return b.done(name="quad")


def merge(*scenes):
    b = _Builder()
    for s in scenes:
        b.add(s["vertices"].astype(np.float64), s["indices"].astype(np.int64), 0)
        b.m[-1] = s["mesh_ids"].astype(np.int64)
    return b.done(name="+".join(s.get("name", "?") for s in scenes))


def triangle_soup(scene) -> np.ndarray:
    """[n_triangles, 3, 3] float32 vertex positions (a plain gather)."""
    return scene["vertices"][scene["indices"].astype(np.int64)]
