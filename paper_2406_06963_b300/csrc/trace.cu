// Visibility tracing entry points (single image): primary G-buffer rays,
// cone-jittered shadow rays (Section 3.1) and radius-bounded cosine-weighted
// AO rays (Section 3.2, Eqs. 1-3).  The per-pixel device code is in
// trace_device.cuh.
#include <cmath>

#include "trace_device.cuh"

namespace dhr {
namespace {

// kStats: also count rays, node visits and triangle tests per ray type into
// stats[0..8] = rays {primary, shadow, AO}, visits {..}, tests {..}.
// kRaster: the primary hit comes from the rasterised keys (raster.cu).
template <bool kHalf, bool kStats = false, bool kRaster = false>
__global__ void __launch_bounds__(128, 10) trace_kernel(SceneView sc, TraceConsts k, void* gbuf_dn,
                                                    uint32_t* gbuf_mesh, uint8_t* mask_out,
                                                    uint8_t* ao_out, unsigned long long* stats = nullptr) {
    trace_pixel<kHalf, kStats, false, false, kRaster>(sc, k, thread_pixel(), gbuf_dn, gbuf_mesh, mask_out, ao_out,
                                                      stats);
}

__global__ void cast_kernel(SceneView sc, const float* orig, const float* dirs, const float* tmin,
                            const float* tmax, int any_hit, int64_t n, float* t_out, int32_t* tri_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Ray r = make_ray(make_float3(orig[3 * i], orig[3 * i + 1], orig[3 * i + 2]),
                          make_float3(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]));
    float tm = tmax[i];
    float3 b;
    const int leaf = any_hit ? traverse<true>(sc, r, tmin[i], tm, b) : traverse<false>(sc, r, tmin[i], tm, b);
    t_out[i] = leaf >= 0 ? tm : INFINITY;
    tri_out[i] = leaf >= 0 ? (int32_t)__float_as_uint(__ldg(sc.tris + 3 * leaf).w) : -1;
}

__global__ void sample_kernel(const uint32_t* px, const uint32_t* py, int64_t n, uint32_t frame,
                              uint32_t seed, uint32_t sample, const float* normals, float3 light,
                              float tan_cone, float* disk_ao, float* dir_ao, float* disk_sh,
                              float* dir_sh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 a = disk_point(px[i], py[i], frame, seed, kAoRay, sample);
    const float3 da = ao_direction(make_float3(normals[3 * i], normals[3 * i + 1], normals[3 * i + 2]), a);
    const float2 s = disk_point(px[i], py[i], frame, seed, kShadowRay, sample);
    const float3 ds = cone_direction(light, tan_cone, s);
    disk_ao[2 * i] = a.x;
    disk_ao[2 * i + 1] = a.y;
    dir_ao[3 * i] = da.x;
    dir_ao[3 * i + 1] = da.y;
    dir_ao[3 * i + 2] = da.z;
    disk_sh[2 * i] = s.x;
    disk_sh[2 * i + 1] = s.y;
    dir_sh[3 * i] = ds.x;
    dir_sh[3 * i + 1] = ds.y;
    dir_sh[3 * i + 2] = ds.z;
}

}  // namespace

// tan of the cone half angle: computed in double on the host, rounded once
static float cone_tan(float angle) { return (float)std::tan((double)angle); }

dhr_status check_trace_params(const dhr_trace_params* p) {
    DHR_CHECK_ARG(p, "trace params: null");
    DHR_CHECK_ARG(p->n_lights >= 1 && p->n_lights <= DHR_MAX_LIGHTS, "n_lights %u not in 1..%d",
                  p->n_lights, DHR_MAX_LIGHTS);
    DHR_CHECK_ARG(p->ao_spp >= 1 && p->ao_spp <= 255, "ao_spp %u not in 1..255", p->ao_spp);
    DHR_CHECK_ARG(p->ao_radius > 0.0f, "ao_radius must be > 0");
    DHR_CHECK_ARG(p->primary == DHR_PRIMARY_TRAVERSE || p->primary == DHR_PRIMARY_RASTER,
                  "primary %u is neither DHR_PRIMARY_TRAVERSE nor DHR_PRIMARY_RASTER", p->primary);
    for (uint32_t l = 0; l < p->n_lights; ++l) {
        DHR_CHECK_ARG(p->cone_half_angle[l] >= 0.0f && p->cone_half_angle[l] < 1.5707963f,
                      "cone_half_angle[%u] not in [0, pi/2)", l);
        const double lx = p->light_dir[l][0], ly = p->light_dir[l][1], lz = p->light_dir[l][2];
        const double n2 = lx * lx + ly * ly + lz * lz;
        DHR_CHECK_ARG(n2 > 0.0 && std::isfinite(n2), "light_dir[%u] is zero or not finite", l);
    }
    return DHR_OK;
}

dhr_status launch_trace(const dhr_scene* sc, const dhr_camera* cam, const dhr_trace_params* p,
                        dhr_gbuffer* g, uint8_t* mask, uint8_t* ao, cudaStream_t st,
                        unsigned long long* stats, cudaEvent_t after_primary) {
    const TraceConsts k = make_trace_consts(*cam, *p);
    const dim3 grid((cam->width + 15) / 16, (cam->height + 7) / 8);
    if (stats) {
        bool raster = false;
        if (p->primary == DHR_PRIMARY_RASTER) DHR_TRY(launch_raster(sc, cam, g, st, &raster));
        if (raster)
            trace_kernel<false, true, true><<<grid, 128, 0, st>>>(sc->view(), k, g->depth_normal, g->mesh_id, mask,
                                                                  ao, stats);
        else
            trace_kernel<false, true><<<grid, 128, 0, st>>>(sc->view(), k, g->depth_normal, g->mesh_id, mask, ao,
                                                            stats);
        DHR_CUDA_TRY(cudaGetLastError());
        return DHR_OK;
    }
    bool raster = false;
    if (p->primary == DHR_PRIMARY_RASTER) DHR_TRY(launch_raster(sc, cam, g, st, &raster));
    if (after_primary) DHR_CUDA_TRY(cudaEventRecord(after_primary, st));
    auto* dn = g->depth_normal;
    if (g->precision == DHR_FP16) {
        if (raster) trace_kernel<true, false, true><<<grid, 128, 0, st>>>(sc->view(), k, dn, g->mesh_id, mask, ao);
        else trace_kernel<true><<<grid, 128, 0, st>>>(sc->view(), k, dn, g->mesh_id, mask, ao);
    } else {
        if (raster) trace_kernel<false, false, true><<<grid, 128, 0, st>>>(sc->view(), k, dn, g->mesh_id, mask, ao);
        else trace_kernel<false><<<grid, 128, 0, st>>>(sc->view(), k, dn, g->mesh_id, mask, ao);
    }
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}

}  // namespace dhr

using namespace dhr;

extern "C" dhr_status dhr_cast_rays(const dhr_scene* scene, const float* origins, const float* dirs,
                                    const float* tmin, const float* tmax, int32_t any_hit, int64_t n,
                                    float* t_out, int32_t* tri_out, void* stream) {
    clear_error();
    DHR_CHECK_ARG(scene, "cast_rays: null scene");
    DHR_CHECK_ARG(n >= 0, "cast_rays: n < 0");
    if (n == 0) return DHR_OK;
    DHR_CHECK_ARG(origins && dirs && tmin && tmax && t_out && tri_out, "cast_rays: null pointer");
    const int64_t blocks = (n + 127) / 128;
    DHR_CHECK_ARG(blocks < (1ll << 31), "cast_rays: n too large");
    cast_kernel<<<(unsigned)blocks, 128, 0, as_stream(stream)>>>(scene->view(), origins, dirs, tmin, tmax,
                                                                 any_hit, n, t_out, tri_out);
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}

extern "C" dhr_status dhr_sample_directions(const uint32_t* px, const uint32_t* py, int64_t n,
                                            uint32_t frame, uint32_t seed, uint32_t sample,
                                            const float* normals, const float* light,
                                            float cone_half_angle, float* disk_ao, float* dir_ao,
                                            float* disk_sh, float* dir_sh, void* stream) {
    clear_error();
    DHR_CHECK_ARG(n >= 0, "sample_directions: n < 0");
    if (n == 0) return DHR_OK;
    DHR_CHECK_ARG(px && py && normals && light && disk_ao && dir_ao && disk_sh && dir_sh,
                  "sample_directions: null pointer");
    float l[3];
    DHR_CUDA_TRY(cudaMemcpyAsync(l, light, sizeof(l), cudaMemcpyDeviceToHost, as_stream(stream)));
    DHR_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    const int64_t blocks = (n + 127) / 128;
    sample_kernel<<<(unsigned)blocks, 128, 0, as_stream(stream)>>>(
        px, py, n, frame, seed, sample, normals, make_float3(l[0], l[1], l[2]), cone_tan(cone_half_angle),
        disk_ao, dir_ao, disk_sh, dir_sh);
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}

extern "C" dhr_status dhr_trace_stats(const dhr_scene* scene, const dhr_camera* cam, const dhr_trace_params* params,
                                      uint64_t* counters, void* stream) {
    clear_error();
    DHR_CHECK_ARG(scene && cam && counters, "trace_stats: null pointer");
    DHR_TRY(check_trace_params(params));
    DHR_CHECK_ARG(cam->width > 0 && cam->height > 0, "trace_stats: bad camera size");
    cudaStream_t st = as_stream(stream);
    const size_t n = (size_t)cam->width * cam->height;
    unsigned long long* d = nullptr;
    void* dn = nullptr;
    uint32_t* mesh = nullptr;
    uint8_t* mb = nullptr;
    cudaError_t e = cudaMalloc(&d, 9 * sizeof(unsigned long long));
    if (!e) e = cudaMalloc(&dn, n * 16);
    if (!e) e = cudaMalloc((void**)&mesh, n * 4);
    if (!e) e = cudaMalloc((void**)&mb, n * 2);
    if (!e) e = cudaMemsetAsync(d, 0, 9 * sizeof(unsigned long long), st);
    dhr_status s = DHR_OK;
    if (!e) {
        dhr_gbuffer g{DHR_FP32, cam->width, cam->height, dn, mesh};
        s = launch_trace(scene, cam, params, &g, mb, mb + n, st, d);
        if (s == DHR_OK) e = cudaMemcpyAsync(counters, d, 9 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (s == DHR_OK && !e) e = cudaStreamSynchronize(st);
    }
    cudaFree(d);
    cudaFree(dn);
    cudaFree(mesh);
    cudaFree(mb);
    if (e) return set_error(DHR_ERR_CUDA, "trace_stats: %s", cudaGetErrorString(e));
    return s;
}

extern "C" dhr_status dhr_trace_timed(const dhr_scene* scene, const dhr_camera* cam, const dhr_trace_params* params,
                                      dhr_gbuffer* gbuf_out, uint8_t* shadow_mask_out, uint8_t* ao_count_out,
                                      float* ms, void* stream) {
    clear_error();
    DHR_CHECK_ARG(ms, "trace_timed: null ms");
    cudaStream_t st = as_stream(stream);
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < 3 && !err; ++i) err = cudaEventCreate(&e[i]);
    dhr_status s = DHR_OK;
    if (!err) err = cudaEventRecord(e[0], st);
    if (!err) {
        s = dhr_trace_visibility_events(scene, cam, params, gbuf_out, shadow_mask_out, ao_count_out, st, e[1]);
        if (s == DHR_OK) err = cudaEventRecord(e[2], st);
    }
    if (s == DHR_OK && !err) err = cudaEventSynchronize(e[2]);
    if (s == DHR_OK && !err) err = cudaEventElapsedTime(&ms[0], e[0], e[1]);
    if (s == DHR_OK && !err) err = cudaEventElapsedTime(&ms[1], e[1], e[2]);
    for (int i = 0; i < 3; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    if (err) return set_error(DHR_ERR_CUDA, "trace_timed: %s", cudaGetErrorString(err));
    return s;
}
