// Selective shadow rays (Section 5: the shadow-map ray mask of Lauterbach and
// Manocha that the paper plans to adopt).  A shadow map per directional light
// is rendered once per scene and light by casting one closest-hit ray per
// texel through the BVH; a min pyramid over it bounds the nearest occluder.
// The selective trace classifies every receiver against the map
// (smap_classify in trace_device.cuh) and casts the light's cone ray only
// where the map cannot decide.
#include <cmath>
#include <cstring>

#include "trace_device.cuh"

struct dhr_shadow_map {
    const dhr_scene* scene = nullptr;
    int32_t res = 0, levels = 0;
    float* data = nullptr;          // all levels (smap_level_offset)
    uint32_t* scratch = nullptr;    // 6 flipped bounds
    double L[3], eu[3], ev[3], u0, v0, w, h;
    float zmin = INFINITY;
    uint64_t bytes = 0;
    float build_ms = 0.f;
};

namespace dhr {
namespace {

__device__ __forceinline__ uint32_t flip_f32(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __forceinline__ float unflip_f32(uint32_t u) {
    const uint32_t v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &v, 4);
    return f;
}

// bounds of every triangle vertex: b[0..2] = flipped min, b[3..5] = flipped max
__global__ void tri_bounds_kernel(const float4* tris, int64_t n3, uint32_t* b) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = __ldg(tris + i);
        lo[0] = fminf(lo[0], v.x);
        lo[1] = fminf(lo[1], v.y);
        lo[2] = fminf(lo[2], v.z);
        hi[0] = fmaxf(hi[0], v.x);
        hi[1] = fmaxf(hi[1], v.y);
        hi[2] = fmaxf(hi[2], v.z);
    }
    for (int o = 16; o; o >>= 1)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 3; ++k) {
            atomicMin(b + k, flip_f32(lo[k]));
            atomicMax(b + 3 + k, flip_f32(hi[k]));
        }
}

struct SmapFrameF {
    float3 L, eu, ev;
    float u0, v0, w, h;
    int res;
};

// one texel per thread: closest hit of the ray from the light plane along -L
__global__ void __launch_bounds__(128) smap_render_kernel(SceneView sc, SmapFrameF f, float* S) {
    const int i = blockIdx.x * 16 + (threadIdx.x & 15), j = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (i >= f.res || j >= f.res) return;
    const float u = f.u0 + ((float)i + 0.5f) * f.w, v = f.v0 + ((float)j + 0.5f) * f.w;
    const float3 o = make_float3(f.h * f.L.x + u * f.eu.x + v * f.ev.x, f.h * f.L.y + u * f.eu.y + v * f.ev.y,
                                 f.h * f.L.z + u * f.eu.z + v * f.ev.z);
    float tm = INFINITY;
    float3 b;
    const int leaf = traverse<false>(sc, make_ray(o, make_float3(-f.L.x, -f.L.y, -f.L.z)), 0.0f, tm, b);
    S[(size_t)j * f.res + i] = leaf >= 0 ? tm : INFINITY;
}

// level l from level l - 1: minimum of 2 x 2 texels
__global__ void smap_min_kernel(const float* in, float* out, int Rl) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)Rl * Rl) return;
    const int i = (int)(k % Rl), j = (int)(k / Rl);
    const float* a = in + (size_t)(2 * j) * (2 * Rl) + 2 * i;
    out[k] = fminf(fminf(a[0], a[1]), fminf(a[2 * Rl], a[2 * Rl + 1]));
}

template <bool kHalf, bool kRaster>
__global__ void __launch_bounds__(128, 10) trace_sel_kernel(SceneView sc, TraceConsts k, const __grid_constant__ SmapSet sel,
                                                        void* gbuf_dn, uint32_t* gbuf_mesh, uint8_t* mask_out,
                                                        uint8_t* ao_out, uint8_t* ray_mask) {
    trace_pixel<kHalf, false, false, true, kRaster>(sc, k, thread_pixel(), gbuf_dn, gbuf_mesh, mask_out, ao_out,
                                                    nullptr, &sel, ray_mask);
}

void cross_d(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
double dot_d(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Frame of the map (double): unit L; helper axis (0,1,0) unless |L.y| >= 0.9,
// then (1,0,0); eu = normalised helper x L, ev = L x eu; the R x R texels of
// size w = E (1 + 2^-10) / R are centred on the projected scene bounds
// (E = the larger projected side); the light plane lies E / 64 above the
// highest bound corner along L.
void make_frame(dhr_shadow_map* m, const float* light, const float lo[3], const float hi[3]) {
    const double l[3] = {light[0], light[1], light[2]};
    const double ln = std::sqrt(dot_d(l, l));
    for (int k = 0; k < 3; ++k) m->L[k] = l[k] / ln;
    double a[3] = {0.0, 0.0, 0.0};
    if (std::fabs(m->L[1]) < 0.9) a[1] = 1.0;
    else a[0] = 1.0;
    double c[3];
    cross_d(a, m->L, c);
    const double cn = std::sqrt(dot_d(c, c));
    for (int k = 0; k < 3; ++k) m->eu[k] = c[k] / cn;
    cross_d(m->L, m->eu, m->ev);
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY, tmax = -INFINITY;
    for (int k = 0; k < 8; ++k) {
        const double p[3] = {(k & 1) ? hi[0] : lo[0], (k & 2) ? hi[1] : lo[1], (k & 4) ? hi[2] : lo[2]};
        const double u = dot_d(m->eu, p), v = dot_d(m->ev, p), t = dot_d(m->L, p);
        umin = std::fmin(umin, u);
        umax = std::fmax(umax, u);
        vmin = std::fmin(vmin, v);
        vmax = std::fmax(vmax, v);
        tmax = std::fmax(tmax, t);
    }
    double E = std::fmax(umax - umin, vmax - vmin);
    if (!(E > 0.0)) E = 1.0;
    m->w = E * (1.0 + 1.0 / 1024.0) / m->res;
    m->u0 = 0.5 * (umin + umax) - 0.5 * m->w * m->res;
    m->v0 = 0.5 * (vmin + vmax) - 0.5 * m->w * m->res;
    m->h = tmax + E / 64.0;
}

SmapFrameF frame_f(const dhr_shadow_map* m) {
    SmapFrameF f;
    f.L = make_float3((float)m->L[0], (float)m->L[1], (float)m->L[2]);
    f.eu = make_float3((float)m->eu[0], (float)m->eu[1], (float)m->eu[2]);
    f.ev = make_float3((float)m->ev[0], (float)m->ev[1], (float)m->ev[2]);
    f.u0 = (float)m->u0;
    f.v0 = (float)m->v0;
    f.w = (float)m->w;
    f.h = (float)m->h;
    f.res = m->res;
    return f;
}

}  // namespace

dhr_status launch_trace_selective(const dhr_scene* sc, const dhr_camera* cam, const dhr_trace_params* p,
                                  const dhr_shadow_map* const* maps, dhr_gbuffer* g, uint8_t* mask, uint8_t* ao,
                                  uint8_t* ray_mask, cudaStream_t st) {
    SmapSet sel;
    for (int l = 0; l < DHR_MAX_LIGHTS; ++l) {
        SmapView& v = sel.m[l];
        v = SmapView{};
        v.S = nullptr;
        const dhr_shadow_map* m = (maps && l < (int)p->n_lights) ? maps[l] : nullptr;
        if (!m) continue;
        DHR_CHECK_ARG(m->scene == sc, "trace_selective: shadow map %d was built for another scene", l);
        const double pl[3] = {p->light_dir[l][0], p->light_dir[l][1], p->light_dir[l][2]};
        const double pn = std::sqrt(dot_d(pl, pl));
        DHR_CHECK_ARG(pn > 0.0 && 1.0 - dot_d(pl, m->L) / pn < 1e-6,
                      "trace_selective: shadow map %d was built for another light direction", l);
        const SmapFrameF f = frame_f(m);
        v.S = m->data;
        v.res = m->res;
        v.L = f.L;
        v.eu = f.eu;
        v.ev = f.ev;
        v.u0 = f.u0;
        v.v0 = f.v0;
        v.w = f.w;
        v.inv_w = (float)(1.0 / m->w);
        v.h = f.h;
        v.zmin = m->zmin;
        const double th = (double)p->cone_half_angle[l];
        v.tau = (float)std::tan(th);
        v.graze = (float)(std::sin(th) + kSmapGraze);
    }
    const TraceConsts k = make_trace_consts(*cam, *p);
    const dim3 grid((cam->width + 15) / 16, (cam->height + 7) / 8);
    bool raster = false;
    if (p->primary == DHR_PRIMARY_RASTER) DHR_TRY(launch_raster(sc, cam, g, st, &raster));
    void* dn = g->depth_normal;
    if (g->precision == DHR_FP16) {
        if (raster) trace_sel_kernel<true, true><<<grid, 128, 0, st>>>(sc->view(), k, sel, dn, g->mesh_id, mask, ao, ray_mask);
        else trace_sel_kernel<true, false><<<grid, 128, 0, st>>>(sc->view(), k, sel, dn, g->mesh_id, mask, ao, ray_mask);
    } else {
        if (raster) trace_sel_kernel<false, true><<<grid, 128, 0, st>>>(sc->view(), k, sel, dn, g->mesh_id, mask, ao, ray_mask);
        else trace_sel_kernel<false, false><<<grid, 128, 0, st>>>(sc->view(), k, sel, dn, g->mesh_id, mask, ao, ray_mask);
    }
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}

}  // namespace dhr

using namespace dhr;

extern "C" dhr_status dhr_shadow_map_create(const dhr_scene* scene, const float* light_dir, int32_t resolution,
                                            void* stream, dhr_shadow_map** out) {
    clear_error();
    DHR_CHECK_ARG(scene && light_dir && out, "shadow_map_create: null pointer");
    *out = nullptr;
    DHR_CHECK_ARG(resolution >= 16 && resolution <= 8192 && (resolution & (resolution - 1)) == 0,
                  "shadow_map_create: resolution %d is not a power of two in 16..8192", resolution);
    const double l2 = (double)light_dir[0] * light_dir[0] + (double)light_dir[1] * light_dir[1] +
                      (double)light_dir[2] * light_dir[2];
    DHR_CHECK_ARG(std::isfinite(l2) && l2 > 0.0, "shadow_map_create: light direction is zero or not finite");
    cudaStream_t st = as_stream(stream);
    dhr_shadow_map* m = new dhr_shadow_map;
    m->scene = scene;
    m->res = resolution;
    m->levels = 1;
    while ((1 << (m->levels - 1)) < resolution) ++m->levels;
    const size_t n_all = smap_level_offset(resolution, m->levels);   // all levels, the last one 1 x 1
    m->bytes = n_all * 4;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void**)&m->data, n_all * 4);
    if (!e) e = cudaMalloc((void**)&m->scratch, 6 * 4);
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    if (!e) e = cudaEventRecord(e0, st);
    float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f};
    if (!e && scene->n_tris > 0) {
        const uint32_t init[6] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u, 0u};
        uint32_t b[6];
        e = cudaMemcpyAsync(m->scratch, init, sizeof(init), cudaMemcpyHostToDevice, st);
        if (!e) {
            tri_bounds_kernel<<<148 * 4, 256, 0, st>>>(scene->tris, 3 * (int64_t)scene->n_tris, m->scratch);
            e = cudaGetLastError();
        }
        if (!e) e = cudaMemcpyAsync(b, m->scratch, sizeof(b), cudaMemcpyDeviceToHost, st);
        if (!e) e = cudaStreamSynchronize(st);
        for (int k = 0; k < 3 && !e; ++k) {
            lo[k] = unflip_f32(b[k]);
            hi[k] = unflip_f32(b[3 + k]);
        }
    }
    if (!e) {
        make_frame(m, light_dir, lo, hi);
        const dim3 grid((resolution + 15) / 16, (resolution + 7) / 8);
        smap_render_kernel<<<grid, 128, 0, st>>>(scene->view(), frame_f(m), m->data);
        e = cudaGetLastError();
        for (int l = 1; l < m->levels && !e; ++l) {
            const int Rl = resolution >> l;
            const int64_t n = (int64_t)Rl * Rl;
            smap_min_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
                m->data + smap_level_offset(resolution, l - 1), m->data + smap_level_offset(resolution, l), Rl);
            e = cudaGetLastError();
        }
    }
    if (!e) e = cudaMemcpyAsync(&m->zmin, m->data + smap_level_offset(resolution, m->levels - 1), 4,
                                cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaEventRecord(e1, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (!e) e = cudaEventElapsedTime(&m->build_ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e) {
        cudaFree(m->data);
        cudaFree(m->scratch);
        delete m;
        return set_error(e == cudaErrorMemoryAllocation ? DHR_ERR_OOM : DHR_ERR_CUDA, "shadow_map_create: %s",
                         cudaGetErrorString(e));
    }
    *out = m;
    return DHR_OK;
}

extern "C" void dhr_shadow_map_destroy(dhr_shadow_map* m) {
    if (!m) return;
    cudaFree(m->data);
    cudaFree(m->scratch);
    delete m;
}

extern "C" dhr_status dhr_shadow_map_get_info(const dhr_shadow_map* m, dhr_shadow_map_info* out) {
    clear_error();
    DHR_CHECK_ARG(m && out, "shadow_map_get_info: null pointer");
    out->resolution = m->res;
    out->levels = m->levels;
    for (int k = 0; k < 3; ++k) {
        out->light_dir[k] = (float)m->L[k];
        out->axis_u[k] = (float)m->eu[k];
        out->axis_v[k] = (float)m->ev[k];
    }
    out->u0 = (float)m->u0;
    out->v0 = (float)m->v0;
    out->texel = (float)m->w;
    out->plane = (float)m->h;
    out->depth_min = m->zmin;
    out->depth = m->data;
    out->bytes = m->bytes;
    out->build_ms = m->build_ms;
    return DHR_OK;
}
