"""ctypes wrapper of the CPU oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline and
reference legs may import this package.  The oracle is plain C in double
precision (binary32 only where a float decides an integer), brute force over
every triangle, and shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_lib = None


def lib():
    """The compiled oracle.  ORC_LIB, when set, names another build of the
    same source to load instead (the pin tests load copies with a planted
    mistake through it and must then fail)."""
    global _lib
    if _lib is None:
        path = os.environ.get("ORC_LIB") or _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


class OrcCamera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("fwd", C.c_float * 3), ("right", C.c_float * 3),
                ("up", C.c_float * 3), ("tan_half_fov_y", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class OrcTraceParams(C.Structure):
    _fields_ = [("n_lights", C.c_int32), ("light_dir", (C.c_float * 3) * 8),
                ("cone_half_angle", C.c_float * 8), ("ao_radius", C.c_float),
                ("ao_spp", C.c_int32), ("frame", C.c_uint32), ("seed", C.c_uint32)]


class OrcMargin(C.Structure):
    _fields_ = [("eps_abs", C.c_double), ("eps_rel", C.c_double)]


class OrcSvgfParams(C.Structure):
    _fields_ = [("alpha", C.c_double), ("sigma_z", C.c_double), ("sigma_n", C.c_double),
                ("sigma_l", C.c_double), ("eps_z", C.c_double), ("eps_l", C.c_double),
                ("ao_spp", C.c_int32), ("levels", C.c_int32), ("fixed_alpha", C.c_int32),
                ("wl_in_atrous", C.c_int32), ("kernel_width", C.c_int32)]


class OrcSmapFrame(C.Structure):
    _fields_ = [("res", C.c_int32), ("L", C.c_double * 3), ("eu", C.c_double * 3), ("ev", C.c_double * 3),
                ("u0", C.c_double), ("v0", C.c_double), ("w", C.c_double), ("h", C.c_double)]


P = C.c_void_p


def _declare(L):
    L.orc_pcg4d.argtypes = [P]
    L.orc_u24.argtypes = [C.c_uint32]
    L.orc_u24.restype = C.c_float
    L.orc_disk_point.argtypes = [C.c_uint32] * 6 + [P]
    L.orc_disk_point.restype = C.c_int
    L.orc_onb_f32.argtypes = [P, P, P]
    L.orc_ao_dir_f32.argtypes = [P, C.c_float, C.c_float, P]
    L.orc_cone_dir_f32.argtypes = [P, C.c_float, C.c_float, C.c_float, P]
    L.orc_sample_batch_f32.argtypes = [C.c_int64, P, P, C.c_uint32, C.c_uint32, C.c_uint32,
                                       P, P, C.c_float, P, P, P, P]
    L.orc_scene_create.argtypes = [P, P, P, C.c_int64, C.c_int64]
    L.orc_scene_create.restype = P
    L.orc_scene_destroy.argtypes = [P]
    L.orc_cast.argtypes = [P, P, P, C.c_double, C.c_double, C.c_int, P, P, P, P, P, P]
    L.orc_trace.argtypes = [P, P, P, P, P, C.c_int64] + [P] * 10
    L.orc_num_threads.restype = C.c_int
    L.orc_svgf_temporal.argtypes = [C.c_int, C.c_int] + [P] * 15
    L.orc_svgf_atrous.argtypes = [C.c_int, C.c_int, P, P, C.c_int, P, P]
    L.orc_svgf_frame.argtypes = [C.c_int, C.c_int] + [P] * 16
    L.orc_svgf_seq_grad.argtypes = [C.c_int, C.c_int, C.c_int] + [P] * 9
    L.orc_delay_warp.argtypes = [C.c_int, C.c_int] + [P] * 11
    L.orc_reproject_check.argtypes = [C.c_int, C.c_int] + [P] * 9
    L.orc_smap_frame_make.argtypes = [P, P, C.c_int32, P]
    L.orc_smap_render.argtypes = [P, P, P, P, C.c_int64, P, P]
    L.orc_smap_classify.argtypes = [P, P, P, C.c_double, C.c_int64, P, P, P, C.c_double, C.c_double, P, P]


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# sampling
# --------------------------------------------------------------------------
def pcg4d(v):
    a = _c(v, np.uint32).copy()
    lib().orc_pcg4d(_p(a))
    return a


def u24(h: int) -> float:
    return lib().orc_u24(int(h))


def disk_point(px, py, frame, seed, ray_type, sample):
    xy = np.zeros(2, np.float32)
    k = lib().orc_disk_point(px, py, frame, seed, ray_type, sample, _p(xy))
    return float(xy[0]), float(xy[1]), k


def onb_f32(n):
    n = _c(n, np.float32)
    T = np.zeros(3, np.float32)
    B = np.zeros(3, np.float32)
    lib().orc_onb_f32(_p(n), _p(T), _p(B))
    return T, B


def ao_dir_f32(n, x, y):
    n = _c(n, np.float32)
    d = np.zeros(3, np.float32)
    lib().orc_ao_dir_f32(_p(n), x, y, _p(d))
    return d


def cone_dir_f32(l, tan_theta, x, y):
    l = _c(l, np.float32)
    d = np.zeros(3, np.float32)
    lib().orc_cone_dir_f32(_p(l), tan_theta, x, y, _p(d))
    return d


def sample_batch(px, py, frame, seed, sample, normals, light, tan_theta):
    px = _c(px, np.uint32)
    py = _c(py, np.uint32)
    n = len(px)
    normals = _c(normals, np.float32).reshape(n, 3)
    light = _c(light, np.float32)
    out = [np.zeros((n, 2), np.float32), np.zeros((n, 3), np.float32),
           np.zeros((n, 2), np.float32), np.zeros((n, 3), np.float32)]
    lib().orc_sample_batch_f32(n, _p(px), _p(py), frame, seed, sample, _p(normals), _p(light),
                               float(np.float32(tan_theta)), *[_p(o) for o in out])
    return dict(disk_ao=out[0], dir_ao=out[1], disk_sh=out[2], dir_sh=out[3])


def tan_f32(angle_rad: float) -> float:
    """tan of the cone half angle, computed in double and rounded once."""
    return float(np.float32(math.tan(float(np.float32(angle_rad)))))


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------
DEFAULT_MARGIN = (1e-6, 1e-6)


class Scene:
    def __init__(self, scene: dict):
        self.v = _c(scene["vertices"], np.float32)
        self.i = _c(scene["indices"], np.uint32)
        self.m = _c(scene["mesh_ids"], np.uint32)
        self.n = len(self.i)
        self.h = lib().orc_scene_create(_p(self.v), _p(self.i), _p(self.m), len(self.v), self.n)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_scene_destroy(self.h)
            self.h = None


def cast(scene: Scene, o, d, tmin=0.0, tmax=math.inf, any_hit=False, margin=DEFAULT_MARGIN):
    o = _c(o, np.float64)
    d = _c(d, np.float64)
    mg = OrcMargin(*margin)
    hit, amb = C.c_int32(), C.c_int32()
    t, tri = C.c_double(), C.c_int64()
    uv = np.zeros(2)
    lib().orc_cast(scene.h, _p(o), _p(d), tmin, tmax, int(any_hit), C.byref(mg), C.byref(hit),
                   C.byref(amb), C.byref(t), C.byref(tri), _p(uv))
    return dict(hit=bool(hit.value), ambiguous=bool(amb.value), t=t.value, tri=tri.value, uv=uv)


def make_camera(cam) -> OrcCamera:
    c = OrcCamera()
    c.pos[:] = [float(x) for x in cam.pos]
    c.fwd[:] = [float(x) for x in cam.forward]
    c.right[:] = [float(x) for x in cam.right]
    c.up[:] = [float(x) for x in cam.up]
    c.tan_half_fov_y = cam.tan_half_fov_y
    c.width = cam.width
    c.height = cam.height
    return c


@dataclass
class TraceParams:
    light_dirs: list = field(default_factory=lambda: [(0.3, 1.0, 0.2)])
    cone_half_angle_deg: list = field(default_factory=lambda: [0.5])
    ao_radius: float = 1.0
    ao_spp: int = 1
    frame: int = 0
    seed: int = 0

    def unit_lights(self):
        """Each direction as binary32, normalised in double, rounded once."""
        out = []
        for l in self.light_dirs:
            l = np.asarray(l, np.float32).astype(np.float64)
            out.append((l / np.linalg.norm(l)).astype(np.float32))
        return out

    def to_c(self) -> OrcTraceParams:
        p = OrcTraceParams()
        ls = self.unit_lights()
        p.n_lights = len(ls)
        for k, l in enumerate(ls):
            p.light_dir[k][:] = [float(x) for x in l]
            p.cone_half_angle[k] = math.radians(self.cone_half_angle_deg[k])
        p.ao_radius = self.ao_radius
        p.ao_spp = self.ao_spp
        p.frame = self.frame
        p.seed = self.seed
        return p


def trace(scene: Scene, cam, params: TraceParams, pixels=None, margin=DEFAULT_MARGIN):
    """Brute-force trace of the given pixels ([n, 2] int (x, y); None = all)."""
    if pixels is None:
        ys, xs = np.mgrid[0:cam.height, 0:cam.width]
        pixels = np.stack([xs.ravel(), ys.ravel()], -1)
    pixels = _c(pixels, np.int32).reshape(-1, 2)
    n = len(pixels)
    out = dict(depth=np.zeros(n), normal=np.zeros((n, 3)), pos=np.zeros((n, 3)),
               tri=np.zeros(n, np.int64), mesh=np.zeros(n, np.uint32),
               shadow_mask=np.zeros(n, np.uint8), ao_count=np.zeros(n, np.uint8),
               amb_primary=np.zeros(n, np.uint8), amb_shadow=np.zeros(n, np.uint8),
               amb_ao=np.zeros(n, np.uint8))
    c = make_camera(cam)
    tp = params.to_c()
    mg = OrcMargin(*margin)
    lib().orc_trace(scene.h, C.byref(c), C.byref(tp), C.byref(mg), _p(pixels), n,
                    *[_p(out[k]) for k in ("depth", "normal", "pos", "tri", "mesh", "shadow_mask",
                                           "ao_count", "amb_primary", "amb_shadow", "amb_ao")])
    out["pixels"] = pixels
    return out


def gbuffer_f32(tr, width, height):
    """Full-frame trace result -> binary32 G-buffer (zn [H, W, 4], mesh [H, W])."""
    zn = np.zeros((height, width, 4), np.float32)
    zn[..., 0] = tr["depth"].reshape(height, width)
    zn[..., 1:] = tr["normal"].reshape(height, width, 3)
    mesh = tr["mesh"].reshape(height, width).astype(np.uint32)
    return zn, mesh


def num_threads() -> int:
    return lib().orc_num_threads()


# --------------------------------------------------------------------------
# modified SVGF
# --------------------------------------------------------------------------
@dataclass
class SvgfParams:
    alpha: float = 0.2
    sigma_z: float = 1.0
    sigma_n: float = 128.0
    sigma_l: float = 4.0
    eps_z: float = 1e-2         # world units: far above the binary32 resolution of depth
    eps_l: float = 1e-3         # far above the binary32 rounding of the colours
    ao_spp: int = 1
    levels: int = 5
    fixed_alpha: bool = False
    wl_in_atrous: bool = True
    kernel_width: int = 5       # 5: 5x5 B3-spline taps; 3: 3x3 (1/4, 1/2, 1/4) taps

    def to_c(self) -> OrcSvgfParams:
        return OrcSvgfParams(self.alpha, self.sigma_z, self.sigma_n, self.sigma_l, self.eps_z,
                             self.eps_l, self.ao_spp, self.levels, int(self.fixed_alpha),
                             int(self.wl_in_atrous), int(self.kernel_width))


class SvgfState:
    """History of the oracle's SVGF: colour, moments, history length."""

    def __init__(self, width, height):
        self.w, self.h = width, height
        self.col = np.zeros((height, width, 2))
        self.mom = np.zeros((height, width, 4))
        self.hist = np.zeros((height, width), np.int32)
        self.prev = None          # (zn, mesh, camera) of the previous frame

    def frame(self, zn, mesh, cam, mask, ao, params: SvgfParams, keep_levels=False):
        W, H = self.w, self.h
        zn = _c(zn, np.float32)
        mesh = _c(mesh, np.uint32)
        mask = _c(mask, np.uint8)
        ao = _c(ao, np.uint8)
        illum = np.zeros((H, W, 4))
        levels = np.zeros((max(params.levels, 1), H, W, 4)) if keep_levels else None
        ao_out = np.zeros((H, W))
        sh_out = np.zeros((H, W))
        c = make_camera(cam)
        if self.prev is not None:
            znp, meshp, camp = self.prev
            cp = make_camera(camp)
        else:
            znp = meshp = None
            cp = c
        pp = params.to_c()
        lib().orc_svgf_frame(W, H, _p(zn), _p(mesh), _p(znp), _p(meshp), C.byref(c), C.byref(cp),
                             _p(mask), _p(ao), C.byref(pp), _p(self.col), _p(self.mom),
                             _p(self.hist), _p(illum), _p(levels), _p(ao_out), _p(sh_out))
        self.prev = (zn, mesh, cam)
        return dict(ao=ao_out, shadow=sh_out, illum=illum, levels=levels)


def svgf_temporal(zn, mesh, cam, mask, ao, params: SvgfParams, prev=None, col_hist=None,
                  mom=None, hist=None):
    """Temporal accumulation + variance only.  prev = (zn, mesh, camera) or None."""
    H, W = zn.shape[:2]
    zn = _c(zn, np.float32)
    mesh = _c(mesh, np.uint32)
    col_hist = _c(col_hist if col_hist is not None else np.zeros((H, W, 2)), np.float64)
    mom = _c(mom if mom is not None else np.zeros((H, W, 4)), np.float64)
    hist = _c(hist if hist is not None else np.zeros((H, W)), np.int32)
    mom_out = np.zeros((H, W, 4))
    hist_out = np.zeros((H, W), np.int32)
    illum = np.zeros((H, W, 4))
    valid = np.zeros((H, W), np.int32)
    c = make_camera(cam)
    if prev is not None:
        znp, meshp = _c(prev[0], np.float32), _c(prev[1], np.uint32)
        cp = make_camera(prev[2])
    else:
        znp = meshp = None
        cp = c
    pp = params.to_c()
    lib().orc_svgf_temporal(W, H, _p(zn), _p(mesh), _p(znp), _p(meshp), C.byref(c), C.byref(cp),
                            _p(_c(mask, np.uint8)), _p(_c(ao, np.uint8)), C.byref(pp),
                            _p(col_hist), _p(mom), _p(hist), _p(mom_out), _p(hist_out), _p(illum),
                            _p(valid))
    return dict(illum=illum, mom=mom_out, hist=hist_out, valid=valid)


def reproject_check(zn, mesh, cam, prev):
    """Reprojection decisions of every pixel taken twice: in binary32 with
    the written operation order the temporal step uses, and in double as
    the plain definition.  prev = (zn, mesh, camera) of the previous frame.
    Returns dec32, dec64 [H,W,4] = (valid, x0, y0, ok bits) and the double
    decision's margins [H,W,4] = (pixels to a bound or the integer grid,
    relative depth to its limit, normal cosine to 0.9, weight sum to
    1e-4)."""
    H, W = zn.shape[:2]
    dec32 = np.zeros((H, W, 4), np.int32)
    dec64 = np.zeros((H, W, 4), np.int32)
    margin = np.zeros((H, W, 4))
    c, cp = make_camera(cam), make_camera(prev[2])
    lib().orc_reproject_check(W, H, _p(_c(zn, np.float32)), _p(_c(mesh, np.uint32)),
                              _p(_c(prev[0], np.float32)), _p(_c(prev[1], np.uint32)), C.byref(c),
                              C.byref(cp), _p(dec32), _p(dec64), _p(margin))
    return dec32, dec64, margin


def svgf_atrous(zn, illum, step, params: SvgfParams):
    H, W = zn.shape[:2]
    zn = _c(zn, np.float32)
    illum = _c(illum, np.float64)
    out = np.zeros((H, W, 4))
    pp = params.to_c()
    lib().orc_svgf_atrous(W, H, _p(zn), _p(illum), int(step), C.byref(pp), _p(out))
    return out


def svgf_seq_grad(zn, mesh, cams, sig, params: SvgfParams, g_out):
    """Forward + hand-derived fp64 adjoint of the SVGF over F frames starting
    without history.  zn [F,H,W,4], mesh [F,H,W], cams (F), sig [F,H,W,2],
    g_out [F,H,W,2].  Returns (out [F,H,W,2], g_sig [F,H,W,2], g_sigma[3]).
    The 5x5 kernel only."""
    if params.kernel_width not in (0, 5):
        raise ValueError("the adjoint is written for the 5x5 kernel")
    zn = _c(zn, np.float32)
    F, H, W = zn.shape[:3]
    mesh = _c(mesh, np.uint32)
    sig = _c(sig, np.float64)
    g_out = _c(g_out, np.float64)
    cam_arr = (OrcCamera * F)(*[make_camera(c) for c in cams])
    out = np.zeros((F, H, W, 2))
    g_sig = np.zeros((F, H, W, 2))
    g_sigma = np.zeros(3)
    pp = params.to_c()
    lib().orc_svgf_seq_grad(F, W, H, _p(zn), _p(mesh), C.cast(cam_arr, C.c_void_p), _p(sig), C.byref(pp),
                            _p(g_out), _p(out), _p(g_sig), _p(g_sigma))
    return out, g_sig, g_sigma


def delay_warp(zn_t, mesh_t, cam_t, zn_s, mesh_s, cam_s, src_ao, src_sh):
    """Warp source-pose values to the target pose (nearest valid pixel, else 1)."""
    H, W = mesh_t.shape
    out_ao, out_sh = np.zeros((H, W)), np.zeros((H, W))
    valid = np.zeros((H, W), np.int32)
    ct, cs = make_camera(cam_t), make_camera(cam_s)
    lib().orc_delay_warp(W, H, _p(_c(zn_t, np.float32)), _p(_c(mesh_t, np.uint32)), C.byref(ct),
                         _p(_c(zn_s, np.float32)), _p(_c(mesh_s, np.uint32)), C.byref(cs),
                         _p(_c(src_ao, np.float64)), _p(_c(src_sh, np.float64)), _p(out_ao), _p(out_sh),
                         _p(valid))
    return out_ao, out_sh, valid


# --------------------------------------------------------------------------
# selective shadow rays (Section 5: shadow-map ray mask)
# --------------------------------------------------------------------------
CLS_TRACE, CLS_LIT, CLS_UMBRA = 0, 1, 2


class ShadowMap:
    """Oracle shadow map of one directional light: the frame (double) and,
    when ``full``, every texel's depth and ambiguity flag (brute force:
    R^2 closest-hit casts over every triangle)."""

    def __init__(self, scene: Scene, light_dir, res: int, full: bool = True, margin=DEFAULT_MARGIN):
        self.light = np.asarray(light_dir, np.float32)      # normalised in double by the oracle
        self.frame = OrcSmapFrame()
        lib().orc_smap_frame_make(scene.h, _p(_c(self.light, np.float32)), int(res), C.byref(self.frame))
        self.res = int(res)
        self.scene = scene
        self.margin = margin
        self.depth = self.amb = None
        if full:
            self.depth = np.zeros((res, res))
            self.amb = np.zeros((res, res), np.uint8)
            mg = OrcMargin(*margin)
            lib().orc_smap_render(scene.h, C.byref(self.frame), C.byref(mg), None, 0, _p(self.depth),
                                  _p(self.amb))

    def frame_dict(self):
        f = self.frame
        return dict(res=f.res, L=np.array(f.L[:]), eu=np.array(f.eu[:]), ev=np.array(f.ev[:]), u0=f.u0,
                    v0=f.v0, w=f.w, h=f.h)

    def texels(self, ij):
        """Depth and ambiguity of the texels ij ([n, 2] int (i, j))."""
        ij = _c(ij, np.int32).reshape(-1, 2)
        d = np.zeros(len(ij))
        a = np.zeros(len(ij), np.uint8)
        mg = OrcMargin(*self.margin)
        lib().orc_smap_render(self.scene.h, C.byref(self.frame), C.byref(mg), _p(ij), len(ij), _p(d), _p(a))
        return d, a

    def classify(self, pos, normal, fg, theta, tol_t=2e-3, tol_z=None):
        """Per-pixel class (CLS_*) and ambiguity flag for cone half angle theta."""
        assert self.depth is not None, "classification needs the full map"
        if tol_z is None:
            tol_z = 1e-5 * (1.0 + self.scene_extent())
        pos = _c(pos, np.float64).reshape(-1, 3)
        normal = _c(normal, np.float64).reshape(-1, 3)
        fg = _c(fg, np.uint8).ravel()
        n = len(pos)
        cls = np.zeros(n, np.uint8)
        amb = np.zeros(n, np.uint8)
        lib().orc_smap_classify(C.byref(self.frame), _p(_c(self.depth, np.float64)), _p(_c(self.amb, np.uint8)),
                                float(theta), n, _p(pos), _p(normal), _p(fg), float(tol_t), float(tol_z),
                                _p(cls), _p(amb))
        return cls, amb

    def scene_extent(self):
        return float(np.abs(self.scene.v).max()) if len(self.scene.v) else 1.0


def trace_selective(scene: Scene, cam, params: TraceParams, maps, pixels=None, margin=DEFAULT_MARGIN):
    """The full trace with each light's shadow bit replaced by its shadow-map
    verdict wherever the classification is LIT (bit 1) or UMBRA (bit 0).
    maps: one ShadowMap (full) or None (trace everywhere) per light.  Adds
    'cls' [n, n_lights], 'amb_cls' [n, n_lights], 'traced' (bit k = light k's
    ray traced) and 'shadow_mask_full' (the full method's bits)."""
    tr = trace(scene, cam, params, pixels, margin)
    n = len(tr["depth"])
    nl = len(params.light_dirs)
    fg = np.isfinite(tr["depth"]).astype(np.uint8)
    cls = np.zeros((n, nl), np.uint8)
    amb = np.zeros((n, nl), np.uint8)
    full = tr["shadow_mask"].copy()
    sel = full.copy()
    traced = np.zeros(n, np.uint8)
    for k in range(nl):
        if maps[k] is None:
            traced |= (fg << k).astype(np.uint8)
            continue
        c, a = maps[k].classify(tr["pos"], tr["normal"], fg, math.radians(params.cone_half_angle_deg[k]))
        cls[:, k], amb[:, k] = c, a
        bit = np.uint8(1 << k)
        sel = np.where((fg == 1) & (c == CLS_LIT), sel | bit, sel)
        sel = np.where((fg == 1) & (c == CLS_UMBRA), sel & ~bit, sel)
        traced |= np.where((fg == 1) & (c == CLS_TRACE), bit, np.uint8(0)).astype(np.uint8)
    tr.update(cls=cls, amb_cls=amb, traced=traced, shadow_mask_full=full, shadow_mask=sel.astype(np.uint8))
    return tr
