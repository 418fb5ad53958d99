"""Python binding of libdhrs (ctypes): argument marshalling only.

Every step of the DHR+S server hot path -- LBVH build, primary/shadow/AO
tracing, modified SVGF -- runs in the CUDA library ``libdhrs.so`` built
in-tree from ``csrc/`` for sm_103a.  PyTorch supplies device memory and
streams.  There is no fallback: if the library is missing or no CUDA
device is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# DHRS_DEBUG=1 in the environment selects the bounds-checked debug build
LIB_PATH = os.path.join(HERE, "libdhrs_debug.so" if os.environ.get("DHRS_DEBUG") == "1" else "libdhrs.so")

DHR_FP32, DHR_FP16 = 0, 1
BACKGROUND = 0xFFFFFFFF
MAX_LIGHTS = 8
PRIMARY_RASTER, PRIMARY_TRAVERSE = 0, 1
TAPE_RECOMPUTE, TAPE_STORE = 0, 1
STATUS = {0: "DHR_OK", 1: "DHR_ERR_INVALID", 2: "DHR_ERR_OOM", 3: "DHR_ERR_CUDA",
          4: "DHR_ERR_TIMEOUT", 5: "DHR_ERR_ADMISSION", 6: "DHR_ERR_STATE"}


class DhrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("forward", C.c_float * 3), ("right", C.c_float * 3),
                ("up", C.c_float * 3), ("tan_half_fov_y", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32)]


BUILD_PLOC, BUILD_LBVH = 0, 1


class SceneDesc(C.Structure):
    _fields_ = [("vertices", C.c_void_p), ("indices", C.c_void_p), ("mesh_ids", C.c_void_p),
                ("n_vertices", C.c_uint32), ("n_triangles", C.c_uint32), ("builder", C.c_uint32)]


class SceneInfo(C.Structure):
    _fields_ = [("n_triangles", C.c_uint32), ("n_nodes", C.c_uint32), ("height", C.c_uint32),
                ("device_bytes", C.c_uint64), ("build_ms", C.c_float)]


class TraceParamsC(C.Structure):
    _fields_ = [("n_lights", C.c_uint32), ("light_dir", (C.c_float * 3) * MAX_LIGHTS),
                ("cone_half_angle", C.c_float * MAX_LIGHTS), ("ao_radius", C.c_float),
                ("ao_spp", C.c_uint32), ("frame", C.c_uint32), ("seed", C.c_uint32),
                ("primary", C.c_uint32)]


class GBufferC(C.Structure):
    _fields_ = [("precision", C.c_int), ("width", C.c_int32), ("height", C.c_int32),
                ("depth_normal", C.c_void_p), ("mesh_id", C.c_void_p)]


class SvgfParamsC(C.Structure):
    _fields_ = [("alpha", C.c_float), ("sigma_z", C.c_float), ("sigma_n", C.c_float),
                ("sigma_l", C.c_float), ("eps_z", C.c_float), ("eps_l", C.c_float),
                ("ao_spp", C.c_uint32), ("levels", C.c_uint32), ("fixed_alpha", C.c_uint32),
                ("wl_in_atrous", C.c_uint32), ("shadow_light", C.c_uint32), ("kernel_width", C.c_uint32)]


class SvgfBuffersC(C.Structure):
    _fields_ = [("illum", C.c_void_p), ("moments", C.c_void_p), ("color_hist", C.c_void_p),
                ("histlen", C.c_void_p)]


_P = C.c_void_p
_SIGNATURES = {
    "dhr_last_error": ([], C.c_char_p),
    "dhr_create_scene": ([_P, _P, _P], C.c_int),
    "dhr_destroy_scene": ([_P], None),
    "dhr_scene_get_info": ([_P, _P], C.c_int),
    "dhr_trace_visibility": ([_P, _P, _P, _P, _P, _P, _P], C.c_int),
    "dhr_cast_rays": ([_P, _P, _P, _P, _P, C.c_int32, C.c_int64, _P, _P, _P], C.c_int),
    "dhr_trace_stats": ([_P, _P, _P, _P, _P], C.c_int),
    "dhr_l2_read_bandwidth": ([C.c_int64, C.c_int32, _P, _P], C.c_int),
    "dhr_debug_status": ([_P, _P], C.c_int),
    "dhr_debug_selftest": ([_P], C.c_int),
    "dhr_trace_timed": ([_P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "dhr_gbuffer_convert": ([_P, _P, _P], C.c_int),
    "dhr_sample_directions": ([_P, _P, C.c_int64, C.c_uint32, C.c_uint32, C.c_uint32, _P, _P,
                               C.c_float, _P, _P, _P, _P, _P], C.c_int),
    "dhr_svgf_create": ([C.c_int32, C.c_int32, C.c_int, _P], C.c_int),
    "dhr_svgf_destroy": ([_P], None),
    "dhr_svgf_get_buffers": ([_P, _P], C.c_int),
    "dhr_svgf_reconstruct": ([_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "dhr_svgf_atrous_noalloc": ([_P, _P, _P, _P, _P, _P], C.c_int),
    "dhr_svgf_tape_create": ([C.c_int32, C.c_int32, C.c_int32, _P], C.c_int),
    "dhr_svgf_tape_destroy": ([_P], None),
    "dhr_svgf_tape_set_schedule": ([_P, C.c_int32], C.c_int),
    "dhr_svgf_tape_level_bytes": ([_P, C.c_int32, _P], C.c_int),
    "dhr_svgf_seq_forward": ([_P, _P, _P, _P, _P, _P, _P], C.c_int),
    "dhr_svgf_seq_backward": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "dhr_delay_warp": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
    "dhr_server_now_ns": ([], C.c_uint64),
    "dhr_server_session_bytes": ([C.c_int32, C.c_int32], C.c_uint64),
    "dhr_server_create": ([_P, C.c_uint64, _P, _P, _P], C.c_int),
    "dhr_server_destroy": ([_P], None),
    "dhr_server_open": ([_P, C.c_int32, C.c_int32, _P], C.c_int),
    "dhr_server_close": ([_P, C.c_int32], C.c_int),
    "dhr_server_submit": ([_P, C.c_int32, _P, _P, C.c_uint32, C.c_uint64, C.c_uint64], C.c_int),
    "dhr_server_set_max_batch_pixels": ([_P, C.c_uint64], C.c_int),
    "dhr_server_set_raster_min_pixels": ([_P, C.c_uint64], C.c_int),
    "dhr_visibility_pack_bound": ([C.c_int32, C.c_int32, C.c_uint32, C.c_uint32], C.c_uint64),
    "dhr_visibility_pack_work": ([C.c_int32, C.c_int32, C.c_uint32, C.c_uint32], C.c_uint64),
    "dhr_visibility_pack": ([_P, _P, C.c_int32, C.c_int32, C.c_uint32, C.c_uint32, _P, _P, _P], C.c_int),
    "dhr_server_pump": ([_P, _P], C.c_int),
    "dhr_server_poll": ([_P, _P, C.c_int32, _P, C.c_int32], C.c_int),
    "dhr_server_output": ([_P, C.c_int32, _P, _P], C.c_int),
    "dhr_server_get_stats": ([_P, _P], C.c_int),
    "dhr_server_read_output": ([_P, C.c_int32, _P, _P], C.c_int),
    "dhr_server_loop_start": ([_P, C.c_uint32, C.c_uint32], C.c_int),
    "dhr_server_loop_stop": ([_P], C.c_int),
    "dhr_server_loop_status": ([_P, _P, _P], C.c_int),
    "dhr_session_create": ([_P, C.c_int32, C.c_int32, C.c_int, _P, _P, _P], C.c_int),
    "dhr_session_destroy": ([_P], None),
    "dhr_step_frame": ([_P, _P, C.c_uint32, _P, _P, _P], C.c_int),
    "dhr_step_frame_host": ([_P, _P, C.c_uint32, _P, _P, _P], C.c_int),
    "dhr_step_frame_host_async": ([_P, _P, C.c_uint32, _P, _P, _P, _P], C.c_int),
    "dhr_session_wait": ([_P, C.c_uint64], C.c_int),
    "dhr_session_get_frame": ([_P, _P, _P, _P], C.c_int),
    "dhr_session_reset": ([_P], C.c_int),
    "dhr_session_checkpoint_bytes": ([_P], C.c_uint64),
    "dhr_session_export": ([_P, _P, C.c_uint64, _P], C.c_int),
    "dhr_session_import": ([_P, _P, C.c_uint64, _P], C.c_int),
    "dhr_shadow_map_create": ([_P, _P, C.c_int32, _P, _P], C.c_int),
    "dhr_shadow_map_destroy": ([_P], None),
    "dhr_shadow_map_get_info": ([_P, _P], C.c_int),
    "dhr_trace_visibility_selective": ([_P, _P, _P, _P, _P, _P, _P, _P, _P], C.c_int),
}

_lib = None


def lib():
    """The loaded libdhrs.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdhrs.so not built ({LIB_PATH}); run "
                               "`python -m paper_2406_06963_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise DhrError(status, lib().dhr_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _need_cuda(*tensors):
    for t in tensors:
        if t is not None and not t.is_cuda:
            raise ValueError("libdhrs expects CUDA tensors")
        if t is not None and not t.is_contiguous():
            raise ValueError("libdhrs expects contiguous tensors")


# --------------------------------------------------------------- structs
def camera(cam) -> Camera:
    """workloads.Camera (or any object with the same fields) -> dhr_camera."""
    c = Camera()
    c.pos[:] = [float(x) for x in cam.pos]
    c.forward[:] = [float(x) for x in cam.forward]
    c.right[:] = [float(x) for x in cam.right]
    c.up[:] = [float(x) for x in cam.up]
    c.tan_half_fov_y = float(cam.tan_half_fov_y)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


@dataclass
class TraceParams:
    light_dirs: list = field(default_factory=lambda: [(0.3, 1.0, 0.2)])
    cone_half_angle_deg: list = field(default_factory=lambda: [0.5])
    ao_radius: float = 1.0
    ao_spp: int = 1
    frame: int = 0
    seed: int = 0
    primary: int = 0        # PRIMARY_RASTER (default) or PRIMARY_TRAVERSE (identical outputs)

    def to_c(self) -> TraceParamsC:
        p = TraceParamsC()
        p.n_lights = len(self.light_dirs)
        for k, l in enumerate(self.light_dirs):
            p.light_dir[k][:] = [float(x) for x in l]       # normalised by the library
            p.cone_half_angle[k] = math.radians(self.cone_half_angle_deg[k])
        p.ao_radius = self.ao_radius
        p.ao_spp = self.ao_spp
        p.frame = self.frame
        p.seed = self.seed
        p.primary = self.primary
        return p


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
    shadow_light: int = 0
    kernel_width: int = 5       # 5: 5x5 B3-spline taps; 3: 3x3 (1/4, 1/2, 1/4) taps

    def to_c(self) -> SvgfParamsC:
        return SvgfParamsC(self.alpha, self.sigma_z, self.sigma_n, self.sigma_l, self.eps_z,
                           self.eps_l, self.ao_spp, self.levels, int(self.fixed_alpha),
                           int(self.wl_in_atrous), int(self.shadow_light), int(self.kernel_width))


# --------------------------------------------------------------- G-buffer
class GBuffer:
    """Device G-buffer + mesh ids [H, W] int32 (bit pattern of the uint32 id).
    FP32: depth_normal float32 [H, W, 4] (depth, normal).  FP16: int32
    [H, W, 2] = (binary32 depth bits, two binary16 octahedral normal
    coordinates) -- use to_fp32() to read it."""

    def __init__(self, width, height, precision=DHR_FP32, device="cuda"):
        import torch
        self.width, self.height, self.precision = width, height, precision
        if precision == DHR_FP16:
            self.depth_normal = torch.empty((height, width, 2), dtype=torch.int32, device=device)
        else:
            self.depth_normal = torch.empty((height, width, 4), dtype=torch.float32, device=device)
        self.mesh = torch.empty((height, width), dtype=torch.int32, device=device)

    @classmethod
    def from_arrays(cls, zn, mesh, precision=DHR_FP32, device="cuda"):
        """Upload a float32 [H, W, 4] G-buffer; FP16 is packed on the device."""
        import torch
        H, W = mesh.shape
        g32 = cls(W, H, DHR_FP32, device)
        g32.depth_normal.copy_(torch.from_numpy(np.ascontiguousarray(zn, np.float32)))
        g32.mesh.copy_(torch.from_numpy(np.ascontiguousarray(mesh).view(np.int32)))
        if precision == DHR_FP32:
            return g32
        return g32.convert(precision)

    def convert(self, precision):
        g = GBuffer(self.width, self.height, precision, self.depth_normal.device)
        a, b = self.c(), g.c()
        _check(lib().dhr_gbuffer_convert(C.byref(a), C.byref(b), _stream(None)))
        return g

    def to_fp32(self):
        return self if self.precision == DHR_FP32 else self.convert(DHR_FP32)

    def c(self) -> GBufferC:
        return GBufferC(self.precision, self.width, self.height, self.depth_normal.data_ptr(),
                        self.mesh.data_ptr())

    def mesh_u32(self) -> np.ndarray:
        return self.mesh.cpu().numpy().view(np.uint32)


# --------------------------------------------------------------- scene
class Scene:
    """Device scene + LBVH built from a host triangle soup (workloads dict)."""

    def __init__(self, scene: dict, stream=None, builder=BUILD_PLOC):
        v = np.ascontiguousarray(scene["vertices"], np.float32)
        i = np.ascontiguousarray(scene["indices"], np.uint32)
        m = np.ascontiguousarray(scene["mesh_ids"], np.uint32)
        d = SceneDesc(v.ctypes.data, i.ctypes.data, m.ctypes.data, len(v), len(i), builder)
        h = C.c_void_p()
        _check(lib().dhr_create_scene(C.byref(d), _stream(stream), C.byref(h)))
        self.h = h

    def info(self) -> dict:
        s = SceneInfo()
        _check(lib().dhr_scene_get_info(self.h, C.byref(s)))
        return dict(n_triangles=s.n_triangles, n_nodes=s.n_nodes, height=s.height,
                    device_bytes=s.device_bytes, build_ms=s.build_ms)

    def close(self):
        if getattr(self, "h", None):
            lib().dhr_destroy_scene(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace_visibility(scene: Scene, cam, params: TraceParams, gbuf: GBuffer, mask, ao, stream=None):
    _need_cuda(gbuf.depth_normal, gbuf.mesh, mask, ao)
    c = camera(cam)
    p = params.to_c()
    g = gbuf.c()
    _check(lib().dhr_trace_visibility(scene.h, C.byref(c), C.byref(p), C.byref(g), _ptr(mask),
                                      _ptr(ao), _stream(stream)))


class ShadowMapInfoC(C.Structure):
    _fields_ = [("resolution", C.c_int32), ("levels", C.c_int32), ("light_dir", C.c_float * 3),
                ("axis_u", C.c_float * 3), ("axis_v", C.c_float * 3), ("u0", C.c_float), ("v0", C.c_float),
                ("texel", C.c_float), ("plane", C.c_float), ("depth_min", C.c_float), ("depth", C.c_void_p),
                ("bytes", C.c_uint64), ("build_ms", C.c_float)]


class ShadowMap:
    """Device shadow map of one directional light over ``scene`` (R x R
    texels plus its min pyramid), for the selective trace."""

    def __init__(self, scene: Scene, light_dir, resolution: int = 4096, stream=None):
        self.light = np.asarray(light_dir, np.float32)   # normalised (or rejected) by the library
        h = C.c_void_p()
        _check(lib().dhr_shadow_map_create(scene.h, self.light.ctypes.data_as(C.c_void_p), int(resolution),
                                           _stream(stream), C.byref(h)))
        self.h = h
        self.scene = scene      # the map must not outlive its scene

    def info(self) -> dict:
        i = ShadowMapInfoC()
        _check(lib().dhr_shadow_map_get_info(self.h, C.byref(i)))
        return dict(resolution=i.resolution, levels=i.levels, light_dir=list(i.light_dir),
                    axis_u=list(i.axis_u), axis_v=list(i.axis_v), u0=i.u0, v0=i.v0, texel=i.texel,
                    plane=i.plane, depth_min=i.depth_min, depth=i.depth, bytes=i.bytes, build_ms=i.build_ms)

    def depth(self):
        """Level 0 as a [R, R] float32 CUDA tensor (a copy)."""
        import torch
        i = self.info()
        R = i["resolution"]
        return torch.as_tensor(_DevArray(i["depth"], (R, R), "<f4"), device="cuda").clone()

    def close(self):
        if getattr(self, "h", None):
            lib().dhr_shadow_map_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace_visibility_selective(scene: Scene, cam, params: TraceParams, maps, gbuf: GBuffer, mask, ao,
                               ray_mask=None, stream=None):
    """trace_visibility with shadow rays only where light k's map (maps[k],
    or None = trace everywhere) cannot decide; ray_mask (uint8 [H, W],
    optional) receives bit k = light k's ray was called for."""
    _need_cuda(gbuf.depth_normal, gbuf.mesh, mask, ao, ray_mask)
    c = camera(cam)
    p = params.to_c()
    g = gbuf.c()
    arr = (C.c_void_p * MAX_LIGHTS)()
    for k, m in enumerate(maps or []):
        arr[k] = m.h.value if m is not None else None
    _check(lib().dhr_trace_visibility_selective(scene.h, C.byref(c), C.byref(p), arr, C.byref(g), _ptr(mask),
                                                _ptr(ao), _ptr(ray_mask), _stream(stream)))


def trace_timed(scene: Scene, cam, params: TraceParams, gbuf: GBuffer, mask, ao, stream=None):
    """trace_visibility timed on the device: (primary pre-pass ms, trace kernel ms)."""
    _need_cuda(gbuf.depth_normal, gbuf.mesh, mask, ao)
    c = camera(cam)
    p = params.to_c()
    g = gbuf.c()
    ms = (C.c_float * 2)()
    _check(lib().dhr_trace_timed(scene.h, C.byref(c), C.byref(p), C.byref(g), _ptr(mask), _ptr(ao), ms,
                                 _stream(stream)))
    return float(ms[0]), float(ms[1])


def trace_stats(scene: Scene, cam, params: TraceParams, stream=None) -> dict:
    """Rays, BVH node visits and triangle tests of one frame, per ray type."""
    c = camera(cam)
    p = params.to_c()
    out = (C.c_uint64 * 9)()
    _check(lib().dhr_trace_stats(scene.h, C.byref(c), C.byref(p), out, _stream(stream)))
    v = list(out)
    return dict(rays=v[0:3], visits=v[3:6], tests=v[6:9])


def l2_read_bandwidth(nbytes: int = 48 << 20, passes: int = 40, stream=None) -> float:
    """Measured L2 read bandwidth (GB/s) of an L2-resident buffer (a
    measurement helper, not a step of the method)."""
    out = C.c_float()
    _check(lib().dhr_l2_read_bandwidth(int(nbytes), int(passes), C.byref(out), _stream(stream)))
    return float(out.value)


def debug_status():
    """(first recorded out-of-bounds event or 0, is_debug_build); the event
    word: bit 63 set, bits 40..47 the site, bits 0..39 the index."""
    err, dbg = C.c_uint64(), C.c_int32()
    _check(lib().dhr_debug_status(C.byref(err), C.byref(dbg)))
    return int(err.value), bool(dbg.value)


def debug_selftest(stream=None):
    """Debug build: one checked out-of-range read that the check records."""
    _check(lib().dhr_debug_selftest(_stream(stream)))


def cast_rays(scene: Scene, origins, dirs, tmin, tmax, any_hit=False, stream=None):
    import torch
    _need_cuda(origins, dirs, tmin, tmax)
    n = origins.shape[0]
    t = torch.empty(n, dtype=torch.float32, device=origins.device)
    tri = torch.empty(n, dtype=torch.int32, device=origins.device)
    _check(lib().dhr_cast_rays(scene.h, _ptr(origins), _ptr(dirs), _ptr(tmin), _ptr(tmax),
                               int(any_hit), n, _ptr(t), _ptr(tri), _stream(stream)))
    return t, tri


def sample_directions(px, py, frame, seed, sample, normals, light, cone_half_angle, stream=None):
    import torch
    _need_cuda(px, py, normals, light)
    n = px.shape[0]
    dev = px.device
    out = dict(disk_ao=torch.empty((n, 2), device=dev), dir_ao=torch.empty((n, 3), device=dev),
               disk_sh=torch.empty((n, 2), device=dev), dir_sh=torch.empty((n, 3), device=dev))
    _check(lib().dhr_sample_directions(_ptr(px), _ptr(py), n, frame, seed, sample, _ptr(normals),
                                       _ptr(light), float(cone_half_angle), _ptr(out["disk_ao"]),
                                       _ptr(out["dir_ao"]), _ptr(out["disk_sh"]),
                                       _ptr(out["dir_sh"]), _stream(stream)))
    return out


# --------------------------------------------------------------- SVGF
class SvgfState:
    def __init__(self, width, height, precision=DHR_FP32):
        h = C.c_void_p()
        _check(lib().dhr_svgf_create(width, height, precision, C.byref(h)))
        self.h, self.width, self.height, self.precision = h, width, height, precision

    def reconstruct(self, cur: GBuffer, prev, cam, cam_prev, mask, ao, params: SvgfParams,
                    ao_out, sh_out, stream=None):
        _need_cuda(mask, ao, ao_out, sh_out)
        c, cp = camera(cam), (camera(cam_prev) if cam_prev is not None else None)
        gc = cur.c()
        gp = prev.c() if prev is not None else None
        p = params.to_c()
        _check(lib().dhr_svgf_reconstruct(self.h, C.byref(gc), C.byref(gp) if gp else None,
                                          C.byref(c), C.byref(cp) if cp else None, _ptr(mask),
                                          _ptr(ao), C.byref(p), _ptr(ao_out), _ptr(sh_out),
                                          _stream(stream)))

    def buffers(self) -> dict:
        """Device pointers of the state's buffers (illum, moments, colour history, histlen)."""
        b = SvgfBuffersC()
        _check(lib().dhr_svgf_get_buffers(self.h, C.byref(b)))
        return dict(illum=b.illum, moments=b.moments, color_hist=b.color_hist, histlen=b.histlen)

    def close(self):
        if getattr(self, "h", None):
            lib().dhr_svgf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevArray:
    """Minimal __cuda_array_interface__ wrapper of a raw device pointer."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = dict(shape=tuple(shape), typestr=typestr, data=(int(ptr), False),
                                             version=2, strides=None)


_TYPESTR = {"float32": "<f4", "float16": "<f2", "uint8": "|u1", "int32": "<i4"}


def svgf_atrous_noalloc(gbuf: GBuffer, illum_ptr: int, params: SvgfParams, ao_out, sh_out, stream=None):
    """A-trous iterations over a float4 illum buffer (device pointer) with the
    library's fixed scratch instead of allocated memory (<= 1,048,576 pixels)."""
    _need_cuda(ao_out, sh_out)
    g = gbuf.c()
    p = params.to_c()
    _check(lib().dhr_svgf_atrous_noalloc(C.byref(g), C.c_void_p(int(illum_ptr)), C.byref(p), _ptr(ao_out),
                                         _ptr(sh_out), _stream(stream)))


def pack_visibility(mask, ao, n_lights: int, ao_spp: int, stream=None):
    """Lossless packed stream (torch uint32 words on the device, trimmed to
    its size) of a frame's bitmask and AO count; the format is in dhrs.h."""
    import torch
    _need_cuda(mask, ao)
    H, W = mask.shape
    bound = lib().dhr_visibility_pack_bound(W, H, n_lights, ao_spp)
    if bound == 0:
        raise DhrError(1, "pack_visibility: bad parameters")
    work = torch.empty(int(lib().dhr_visibility_pack_work(W, H, n_lights, ao_spp)) + 256, dtype=torch.uint8,
                       device=mask.device)
    wp = (work.data_ptr() + 255) & ~255
    out = torch.empty(int(bound) // 4, dtype=torch.int32, device=mask.device)
    _check(lib().dhr_visibility_pack(_ptr(mask), _ptr(ao), W, H, n_lights, ao_spp, C.c_void_p(wp), _ptr(out),
                                     _stream(stream)))
    n_mixed = int(out[4].item())
    T = ((W + 31) // 32) * ((H + 7) // 8)
    planes = n_lights + int(ao_spp).bit_length()
    n_words = 5 + (planes * T + 15) // 16 + 8 * n_mixed
    return out[:n_words]


def device_copy(ptr: int, shape, dtype: str):
    """Copy a library-owned device buffer into a new torch tensor."""
    import torch
    torch.cuda.synchronize()
    return torch.as_tensor(_DevArray(ptr, shape, _TYPESTR[dtype]), device="cuda").clone()


# --------------------------------------------------------------- session
class Session:
    """trace + SVGF per frame with library-owned buffers (dhr_step_frame)."""

    def __init__(self, scene: Scene, width, height, precision=DHR_FP32, trace=None, svgf=None):
        self.trace = trace or TraceParams()
        self.svgf = svgf or SvgfParams(ao_spp=self.trace.ao_spp)
        h = C.c_void_p()
        tp, sp = self.trace.to_c(), self.svgf.to_c()
        _check(lib().dhr_session_create(scene.h, width, height, precision, C.byref(tp), C.byref(sp),
                                        C.byref(h)))
        self.h, self.scene = h, scene
        self.width, self.height, self.precision = width, height, precision

    def step(self, cam, frame, ao_out=None, sh_out=None, stream=None):
        _need_cuda(ao_out, sh_out)
        c = camera(cam)
        _check(lib().dhr_step_frame(self.h, C.byref(c), frame, _ptr(ao_out), _ptr(sh_out),
                                    _stream(stream)))

    def step_host(self, cam, frame, ao_host, sh_host, stream=None):
        """Host-output step; ao_host/sh_host: CPU tensors (pinned for speed)."""
        c = camera(cam)
        _check(lib().dhr_step_frame_host(self.h, C.byref(c), frame, C.c_void_p(ao_host.data_ptr()),
                                         C.c_void_p(sh_host.data_ptr()), _stream(stream)))

    def step_host_async(self, cam, frame, ao_host, sh_host, stream=None) -> int:
        """Streaming host-output step: enqueues the frame and the copy of its
        results into ao_host / sh_host (pinned CPU tensors) and returns a
        ticket; the tensors are valid after wait(ticket)."""
        c = camera(cam)
        t = C.c_uint64()
        _check(lib().dhr_step_frame_host_async(self.h, C.byref(c), frame, C.c_void_p(ao_host.data_ptr()),
                                               C.c_void_p(sh_host.data_ptr()), _stream(stream), C.byref(t)))
        return t.value

    def wait(self, ticket: int):
        _check(lib().dhr_session_wait(self.h, C.c_uint64(ticket)))

    def frame_buffers(self) -> dict:
        g = GBufferC()
        m, a = C.c_void_p(), C.c_void_p()
        _check(lib().dhr_session_get_frame(self.h, C.byref(g), C.byref(m), C.byref(a)))
        return dict(depth_normal=g.depth_normal, mesh=g.mesh_id, mask=m.value, ao=a.value)

    def checkpoint(self, stream=None) -> np.ndarray:
        """The session's history as a host byte image (dhr_session_export)."""
        n = int(lib().dhr_session_checkpoint_bytes(self.h))
        buf = np.empty(n, np.uint8)
        _check(lib().dhr_session_export(self.h, buf.ctypes.data_as(C.c_void_p), n, _stream(stream)))
        return buf

    def restore(self, image: np.ndarray, stream=None):
        """Continue from a checkpoint of a session of the same size and
        precision (dhr_session_import)."""
        image = np.ascontiguousarray(image, dtype=np.uint8)
        _check(lib().dhr_session_import(self.h, image.ctypes.data_as(C.c_void_p), int(image.size), _stream(stream)))

    def reset(self):
        _check(lib().dhr_session_reset(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().dhr_session_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------- adjoint
class SvgfTape:
    """Recording of the differentiable SVGF over F frames (FP32).

    schedule TAPE_RECOMPUTE (default): one frame of a-trous level records,
    earlier frames' levels recomputed by the backward; TAPE_STORE: every
    frame's level records kept by the forward."""

    def __init__(self, width, height, frames, schedule=None):
        h = C.c_void_p()
        _check(lib().dhr_svgf_tape_create(width, height, frames, C.byref(h)))
        self.h, self.width, self.height, self.frames = h, width, height, frames
        if schedule is not None:
            self.set_schedule(schedule)

    def set_schedule(self, schedule):
        _check(lib().dhr_svgf_tape_set_schedule(self.h, int(schedule)))

    def level_bytes(self, levels):
        """Bytes of level records a forward with `levels` levels keeps."""
        b = C.c_int64()
        _check(lib().dhr_svgf_tape_level_bytes(self.h, int(levels), C.byref(b)))
        return b.value

    @staticmethod
    def _arrays(gbufs, cams):
        g = (GBufferC * len(gbufs))(*[x.c() for x in gbufs])
        c = (Camera * len(cams))(*[camera(x) for x in cams])
        return g, c

    def forward(self, gbufs, cams, sig, params: SvgfParams, stream=None):
        """sig: CUDA float32 [F, 2, H, W] -> filtered [F, 2, H, W]."""
        import torch
        _need_cuda(sig)
        out = torch.empty_like(sig)
        g, c = self._arrays(gbufs, cams)
        p = params.to_c()
        _check(lib().dhr_svgf_seq_forward(self.h, g, c, _ptr(sig), C.byref(p), _ptr(out), _stream(stream)))
        return out

    def backward(self, gbufs, cams, sig, params: SvgfParams, g_out, stream=None):
        """-> (dL/d sig [F, 2, H, W], dL/d (sigma_z, sigma_n, sigma_l) [3])."""
        import torch
        g_out = g_out.contiguous()
        _need_cuda(sig, g_out)
        g_sig = torch.empty_like(sig)
        g_sigma = torch.empty(3, dtype=torch.float32, device=sig.device)
        g, c = self._arrays(gbufs, cams)
        p = params.to_c()
        _check(lib().dhr_svgf_seq_backward(self.h, g, c, _ptr(sig), C.byref(p), _ptr(g_out), _ptr(g_sig),
                                           _ptr(g_sigma), _stream(stream)))
        return g_sig, g_sigma

    def close(self):
        if getattr(self, "h", None):
            lib().dhr_svgf_tape_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _svgf_function():
    import torch

    class SVGFSequence(torch.autograd.Function):
        """out = SVGF(sig; sigma_z, sigma_n, sigma_l) over a frame sequence;
        backward = the hand-written CUDA adjoint (levels recomputed)."""

        @staticmethod
        def forward(ctx, sig, sigmas, gbufs, cams, params, tape):
            sz, sn, sl = [float(v) for v in sigmas.detach().cpu()]
            p = SvgfParams(**{**params.__dict__, "sigma_z": sz, "sigma_n": sn, "sigma_l": sl})
            sig_c = sig.detach().contiguous()
            out = tape.forward(gbufs, cams, sig_c, p)
            ctx.tape, ctx.gbufs, ctx.cams, ctx.p, ctx.sig = tape, gbufs, cams, p, sig_c
            ctx.sigmas_meta = (sigmas.dtype, sigmas.device)
            return out

        @staticmethod
        def backward(ctx, g_out):
            g_sig, g_sigma = ctx.tape.backward(ctx.gbufs, ctx.cams, ctx.sig, ctx.p, g_out)
            dt, dev = ctx.sigmas_meta
            return g_sig, g_sigma.to(device=dev, dtype=dt), None, None, None, None

    return SVGFSequence


_SVGF_FN = None


def svgf_sequence(sig, sigmas, gbufs, cams, params: SvgfParams = None, tape: SvgfTape = None):
    """Differentiable SVGF: sig [F, 2, H, W] (CUDA float32, may require grad),
    sigmas [3] = (sigma_z, sigma_n, sigma_l) (may require grad)."""
    global _SVGF_FN
    if _SVGF_FN is None:
        _SVGF_FN = _svgf_function()
    F, _, H, W = sig.shape
    tape = tape or SvgfTape(W, H, F)
    return _SVGF_FN.apply(sig, sigmas, gbufs, cams, params or SvgfParams(), tape)


# --------------------------------------------------------------- serving
class Completion(C.Structure):
    _fields_ = [("request_id", C.c_uint64), ("session", C.c_int32), ("frame", C.c_uint32),
                ("t_arrival_ns", C.c_uint64), ("t_start_ns", C.c_uint64), ("t_done_ns", C.c_uint64),
                ("batch_size", C.c_uint32), ("dropped", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("used_bytes", C.c_uint64), ("open_sessions", C.c_int32),
                ("batches", C.c_uint64), ("frames", C.c_uint64), ("dropped", C.c_uint64)]


def delay_warp(target: GBuffer, cam_target, source: GBuffer, cam_source, src_ao, src_sh, out_ao, out_sh,
               stream=None):
    _need_cuda(src_ao, src_sh, out_ao, out_sh)
    t, s_ = target.c(), source.c()
    ct, cs = camera(cam_target), camera(cam_source)
    _check(lib().dhr_delay_warp(C.byref(t), C.byref(ct), C.byref(s_), C.byref(cs), _ptr(src_ao), _ptr(src_sh),
                                _ptr(out_ao), _ptr(out_sh), _stream(stream)))


def now_ns() -> int:
    return int(lib().dhr_server_now_ns())


def session_bytes(width, height) -> int:
    return int(lib().dhr_server_session_bytes(width, height))


class Server:
    """Continuous-batching server of many sessions (dhr_server_*)."""

    def __init__(self, scene: Scene, budget_bytes, trace=None, svgf=None):
        self.trace = trace or TraceParams()
        self.svgf = svgf or SvgfParams(ao_spp=self.trace.ao_spp)
        h = C.c_void_p()
        tp, sp = self.trace.to_c(), self.svgf.to_c()
        _check(lib().dhr_server_create(scene.h, int(budget_bytes), C.byref(tp), C.byref(sp), C.byref(h)))
        self.h, self.scene = h, scene
        self._buf = (Completion * 4096)()

    def open(self, width, height) -> int:
        sid = C.c_int32()
        _check(lib().dhr_server_open(self.h, width, height, C.byref(sid)))
        return sid.value

    def close_session(self, sid):
        _check(lib().dhr_server_close(self.h, sid))

    def submit(self, sid, cam, frame, t_arrival_ns, request_id, cam_target=None):
        c = camera(cam)
        ct = camera(cam_target) if cam_target is not None else None
        _check(lib().dhr_server_submit(self.h, sid, C.byref(c), C.byref(ct) if ct else None, frame,
                                       int(t_arrival_ns), int(request_id)))

    def set_max_batch_pixels(self, max_pixels: int):
        """Pixel cap of one batch (0: none)."""
        _check(lib().dhr_server_set_max_batch_pixels(self.h, C.c_uint64(max_pixels)))

    def set_raster_min_pixels(self, min_pixels: int):
        """Sessions of at least min_pixels rasterise their primary visibility
        (0: all, 2**64 - 1: none); the G-buffers are the same either way."""
        _check(lib().dhr_server_set_raster_min_pixels(self.h, C.c_uint64(int(min_pixels))))

    def pump(self) -> int:
        n = C.c_int32()
        _check(lib().dhr_server_pump(self.h, C.byref(n)))
        return n.value

    def poll(self, wait=False):
        n = C.c_int32()
        _check(lib().dhr_server_poll(self.h, self._buf, len(self._buf), C.byref(n), int(wait)))
        out = []
        for i in range(n.value):
            c = self._buf[i]
            out.append(dict(request_id=c.request_id, session=c.session, frame=c.frame, t_arrival_ns=c.t_arrival_ns,
                            t_start_ns=c.t_start_ns, t_done_ns=c.t_done_ns, batch_size=c.batch_size,
                            dropped=bool(c.dropped)))
        return out

    def output(self, sid, width, height):
        """Host copies (numpy float32 [H, W]) of the session's last completed
        (warped) AO and shadow, made on the server's own stream (so that it
        does not wait for a running device loop)."""
        a = np.empty((height, width), np.float32)
        b = np.empty((height, width), np.float32)
        _check(lib().dhr_server_read_output(self.h, sid, a.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p)))
        return a, b

    def loop_start(self, idle_ms: int = 1000, max_run_ms: int = 600000):
        """Start the device-resident request loop (dhr_server_loop_start)."""
        _check(lib().dhr_server_loop_start(self.h, int(idle_ms), int(max_run_ms)))

    def loop_stop(self):
        """End the device loop and wait for it; raises DhrError(status 4) if it
        had already ended at its idle or run-time limit."""
        _check(lib().dhr_server_loop_stop(self.h))

    def loop_status(self):
        r, b = C.c_int32(), C.c_uint64()
        _check(lib().dhr_server_loop_status(self.h, C.byref(r), C.byref(b)))
        return bool(r.value), int(b.value)

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().dhr_server_get_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().dhr_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
