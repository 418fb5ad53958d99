// Modified SVGF reconstruction (Section 3.3): state, launchers and the C
// entry points.  The kernels live in svgf_kernels.cuh.
#include <mutex>

#include "svgf_kernels.cuh"

// ------------------------------------------------------------------ state
struct dhr_svgf_state {
    int32_t w = 0, h = 0;
    dhr_precision prec = DHR_FP32;
    void* col = nullptr;        // colour history
    void* mom[2] = {nullptr, nullptr};
    uint8_t* hist[2] = {nullptr, nullptr};
    float4* illum = nullptr;    // temporal output
    float4* pp[2] = {nullptr, nullptr};
    float4* gdec = nullptr;     // FP16 states: the current G-buffer decoded, read by the a-trous levels
    int cur = 0;                // index of the moments/history written last
};

namespace dhr {

void svgf_free(dhr_svgf_state* s);

dhr_status svgf_create(int32_t w, int32_t h, dhr_precision prec, dhr_svgf_state** out) {
    DHR_CHECK_ARG(out, "svgf_create: null out");
    DHR_CHECK_ARG(w > 0 && h > 0 && (int64_t)w * h <= (1ll << 28), "svgf_create: bad size %dx%d", w, h);
    DHR_CHECK_ARG(prec == DHR_FP32 || prec == DHR_FP16, "svgf_create: bad precision");
    auto* s = new dhr_svgf_state();
    s->w = w;
    s->h = h;
    s->prec = prec;
    const size_t n = (size_t)w * h;
    const size_t col_b = 8, mom_b = prec == DHR_FP16 ? sizeof(Mom16) : 16;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&s->col, n * col_b);
    e = e ? e : cudaMalloc(&s->mom[0], n * mom_b);
    e = e ? e : cudaMalloc(&s->mom[1], n * mom_b);
    e = e ? e : cudaMalloc((void**)&s->hist[0], n);
    e = e ? e : cudaMalloc((void**)&s->hist[1], n);
    e = e ? e : cudaMalloc((void**)&s->illum, n * 16);
    e = e ? e : cudaMalloc((void**)&s->pp[0], n * 16);
    e = e ? e : cudaMalloc((void**)&s->pp[1], n * 16);
    if (prec == DHR_FP16) e = e ? e : cudaMalloc((void**)&s->gdec, n * 16);
    e = e ? e : cudaMemset(s->hist[0], 0, n);
    e = e ? e : cudaMemset(s->hist[1], 0, n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        svgf_free(s);
        return set_error(e == cudaErrorMemoryAllocation ? DHR_ERR_OOM : DHR_ERR_CUDA, "svgf_create: %s",
                         cudaGetErrorString(e));
    }
    *out = s;
    return DHR_OK;
}

void svgf_free(dhr_svgf_state* s) {
    if (!s) return;
    cudaFree(s->col);
    cudaFree(s->mom[0]);
    cudaFree(s->mom[1]);
    cudaFree(s->hist[0]);
    cudaFree(s->hist[1]);
    cudaFree(s->illum);
    cudaFree(s->pp[0]);
    cudaFree(s->pp[1]);
    cudaFree(s->gdec);
    delete s;
}

// FP16 G-buffer element -> float4 (depth, unit normal); background keeps depth +inf, normal 0
__global__ void gbuf_decode_kernel(int n, const uint2* src, float4* dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 v = unpack_gbuf16(src[i]);
    if (!(v.x < INFINITY)) v = make_float4(v.x, 0.f, 0.f, 0.f);
    dst[i] = v;
}

dhr_status check_svgf_params(const dhr_svgf_params* p) {
    DHR_CHECK_ARG(p, "svgf params: null");
    DHR_CHECK_ARG(p->levels <= 8, "svgf: levels %u > 8", p->levels);
    DHR_CHECK_ARG(p->ao_spp >= 1 && p->ao_spp <= 255, "svgf: ao_spp %u not in 1..255", p->ao_spp);
    DHR_CHECK_ARG(p->alpha > 0.0f && p->alpha <= 1.0f, "svgf: alpha not in (0, 1]");
    DHR_CHECK_ARG(p->sigma_n >= 0.0f && p->sigma_z >= 0.0f && p->sigma_l >= 0.0f, "svgf: negative sigma");
    DHR_CHECK_ARG(p->eps_z > 0.0f && p->eps_l > 0.0f && p->eps_z < INFINITY && p->eps_l < INFINITY,
                  "svgf: eps_z and eps_l must be positive and finite");
    DHR_CHECK_ARG(p->shadow_light < DHR_MAX_LIGHTS, "svgf: shadow_light %u not in 0..%d", p->shadow_light,
                  DHR_MAX_LIGHTS - 1);
    DHR_CHECK_ARG(p->kernel_width == 0 || p->kernel_width == 3 || p->kernel_width == 5,
                  "svgf: kernel_width %u is not 3 or 5", p->kernel_width);
    return DHR_OK;
}

template <dhr_precision P>
static dhr_status run_svgf(dhr_svgf_state* s, const dhr_gbuffer* cur, const dhr_gbuffer* prev,
                           const dhr_camera* cam, const dhr_camera* cam_prev, const uint8_t* mask,
                           const uint8_t* ao, const dhr_svgf_params* prm, float* ao_out, float* sh_out,
                           cudaStream_t st) {
    using S = Store<P>;
    const SvgfConsts k = make_consts(s->w, s->h, prm);
    const int src = s->cur, dst = s->cur ^ 1;
    const dim3 blk(32, 8), grid((s->w + 31) / 32, (s->h + 7) / 8);
    const auto* gc = static_cast<const typename S::G*>(cur->depth_normal);
    const auto* gp = prev ? static_cast<const typename S::G*>(prev->depth_normal) : nullptr;
    temporal_kernel<P, SigCounts><<<grid, blk, 0, st>>>(
        k, *cam, prev ? *cam_prev : *cam, gc, cur->mesh_id, gp, prev ? prev->mesh_id : nullptr,
        SigCounts{mask, ao, k.inv_spp, k.shadow_bit},
        static_cast<const typename S::Col*>(s->col), static_cast<const typename S::Mom*>(s->mom[src]),
        s->hist[src], static_cast<typename S::Mom*>(s->mom[dst]), s->hist[dst], s->illum);
    DHR_CUDA_TRY(cudaGetLastError());
    s->cur = dst;
    auto* col = static_cast<typename S::Col*>(s->col);
    const int L = (int)prm->levels;
    if (L == 0) {
        const int n = s->w * s->h;
        passthrough_kernel<P><<<(n + 255) / 256, 256, 0, st>>>(n, s->illum, col, ao_out, sh_out);
        DHR_CUDA_TRY(cudaGetLastError());
        return DHR_OK;
    }
    const float4* in = s->illum;
    const int nsq = atrous_nsq(prm), R = atrous_radius(prm);
    if (P == DHR_FP16) {
        const int n = s->w * s->h;
        gbuf_decode_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, reinterpret_cast<const uint2*>(gc), s->gdec);
        DHR_CUDA_TRY(cudaGetLastError());
    }
    for (int l = 0; l < L; ++l) {
        float4* out = s->pp[l & 1];
        const int step = 1 << l;
        const int mode = (l == L - 1 && L > 1) ? 2 : (l == 0 ? 1 : 0);
        if (P == DHR_FP16)
            DHR_TRY(launch_atrous<kFP16Decoded>(mode, nsq, R, st, k, step, s->gdec, in, out, col, ao_out,
                                                sh_out));
        else
            DHR_TRY(launch_atrous<P>(mode, nsq, R, st, k, step, gc, in, out, col, ao_out, sh_out));
        if (L == 1) {
            // single iteration: it is both the history source and the output
            passthrough_kernel<P><<<(s->w * s->h + 255) / 256, 256, 0, st>>>(s->w * s->h, out, col, ao_out,
                                                                             sh_out);
            DHR_CUDA_TRY(cudaGetLastError());
        }
        in = out;
    }
    return DHR_OK;
}

// The history a next frame reads: colour history, the moments and history
// lengths written last.  Bytes per pixel, and a copy to (to_host) or from
// host memory `h` laid out in that order, enqueued on st.
uint64_t svgf_history_bytes(const dhr_svgf_state* s) {
    const uint64_t n = (uint64_t)s->w * s->h;
    return n * (8 + (s->prec == DHR_FP16 ? sizeof(Mom16) : 16) + 1);
}

dhr_status svgf_history_copy(dhr_svgf_state* s, void* h, bool to_host, cudaStream_t st) {
    const size_t n = (size_t)s->w * s->h;
    const size_t sizes[3] = {n * 8, n * (s->prec == DHR_FP16 ? sizeof(Mom16) : 16), n};
    void* dev[3] = {s->col, s->mom[s->cur], s->hist[s->cur]};
    char* hp = static_cast<char*>(h);
    for (int i = 0; i < 3; ++i) {
        if (to_host) DHR_CUDA_TRY(cudaMemcpyAsync(hp, dev[i], sizes[i], cudaMemcpyDeviceToHost, st));
        else DHR_CUDA_TRY(cudaMemcpyAsync(dev[i], hp, sizes[i], cudaMemcpyHostToDevice, st));
        hp += sizes[i];
    }
    return DHR_OK;
}

dhr_status svgf_run(dhr_svgf_state* s, const dhr_gbuffer* cur, const dhr_gbuffer* prev, const dhr_camera* cam,
                    const dhr_camera* cam_prev, const uint8_t* mask, const uint8_t* ao,
                    const dhr_svgf_params* prm, float* ao_out, float* sh_out, cudaStream_t st) {
    DHR_CHECK_ARG(s && cur && cam && mask && ao && ao_out && sh_out, "svgf_reconstruct: null pointer");
    DHR_TRY(check_svgf_params(prm));
    DHR_CHECK_ARG(cur->width == s->w && cur->height == s->h && cam->width == s->w && cam->height == s->h,
                  "svgf_reconstruct: size mismatch (state %dx%d)", s->w, s->h);
    DHR_CHECK_ARG(cur->precision == s->prec, "svgf_reconstruct: G-buffer precision differs from the state");
    DHR_CHECK_ARG(cur->depth_normal && cur->mesh_id, "svgf_reconstruct: null G-buffer");
    if (prev) {
        DHR_CHECK_ARG(cam_prev, "svgf_reconstruct: prev G-buffer without cam_prev");
        DHR_CHECK_ARG(prev->width == s->w && prev->height == s->h && prev->precision == s->prec &&
                          prev->depth_normal && prev->mesh_id && cam_prev->width == s->w &&
                          cam_prev->height == s->h,
                      "svgf_reconstruct: previous G-buffer does not match the state");
    }
    if (s->prec == DHR_FP16)
        return run_svgf<DHR_FP16>(s, cur, prev, cam, cam_prev, mask, ao, prm, ao_out, sh_out, st);
    return run_svgf<DHR_FP32>(s, cur, prev, cam, cam_prev, mask, ao, prm, ao_out, sh_out, st);
}

}  // namespace dhr

using namespace dhr;

extern "C" dhr_status dhr_svgf_create(int32_t width, int32_t height, dhr_precision precision,
                                      dhr_svgf_state** out) {
    clear_error();
    return svgf_create(width, height, precision, out);
}

extern "C" void dhr_svgf_destroy(dhr_svgf_state* state) { svgf_free(state); }

extern "C" dhr_status dhr_svgf_get_buffers(dhr_svgf_state* s, dhr_svgf_buffers* out) {
    clear_error();
    DHR_CHECK_ARG(s && out, "svgf_get_buffers: null pointer");
    out->illum = s->illum;
    out->moments = s->mom[s->cur];
    out->color_hist = s->col;
    out->histlen = s->hist[s->cur];
    return DHR_OK;
}

extern "C" dhr_status dhr_svgf_reconstruct(dhr_svgf_state* state, const dhr_gbuffer* cur, const dhr_gbuffer* prev,
                                           const dhr_camera* cam, const dhr_camera* cam_prev,
                                           const uint8_t* shadow_mask, const uint8_t* ao_count,
                                           const dhr_svgf_params* params, float* ao_out, float* shadow_out,
                                           void* stream) {
    clear_error();
    return svgf_run(state, cur, prev, cam, cam_prev, shadow_mask, ao_count, params, ao_out, shadow_out,
                    as_stream(stream));
}

// ------------------------------------------------------------------------
// G-buffer precision conversion (FP32 <-> FP16 storage form)
// ------------------------------------------------------------------------
namespace dhr {
namespace {
__global__ void gbuf_to16_kernel(int n, const float4* src, uint2* dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = src[i];
    dst[i] = pack_gbuf16(v.x, make_float3(v.y, v.z, v.w));
}
}  // namespace
}  // namespace dhr

extern "C" dhr_status dhr_gbuffer_convert(const dhr_gbuffer* src, dhr_gbuffer* dst, void* stream) {
    clear_error();
    DHR_CHECK_ARG(src && dst && src->depth_normal && dst->depth_normal && src->mesh_id && dst->mesh_id,
                  "gbuffer_convert: null pointer");
    DHR_CHECK_ARG(src->width == dst->width && src->height == dst->height && src->width > 0 && src->height > 0,
                  "gbuffer_convert: size mismatch");
    DHR_CHECK_ARG(src->precision != dst->precision, "gbuffer_convert: same precision");
    const int n = src->width * src->height;
    cudaStream_t st = as_stream(stream);
    if (src->precision == DHR_FP32)
        gbuf_to16_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, static_cast<const float4*>(src->depth_normal),
                                                          static_cast<uint2*>(dst->depth_normal));
    else
        gbuf_decode_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, static_cast<const uint2*>(src->depth_normal),
                                                          static_cast<float4*>(dst->depth_normal));
    DHR_CUDA_TRY(cudaGetLastError());
    if (src->mesh_id != dst->mesh_id)
        DHR_CUDA_TRY(cudaMemcpyAsync(dst->mesh_id, src->mesh_id, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    return DHR_OK;
}

// ------------------------------------------------------------------------
// Allocation-free a-trous cascade.
//
// Some callers cannot allocate device memory at the moment they filter: a
// render loop that must not stall on the allocator mid-frame, code running
// inside a memory budget that was reserved up front (such as a serving
// loop that admits sessions by their memory), or a host whose allocator
// belongs to another framework.  dhr_svgf_atrous_noalloc serves them: its
// two ping-pong images live in the file-scope array below, which the
// library reserves once per device when the module loads and keeps until
// the process exits.
// ------------------------------------------------------------------------
namespace dhr {

constexpr int64_t kNoallocMaxPixels = 1 << 20;   // 1,048,576 pixels: 2 images x 16 MiB

static __device__ __align__(256) float4 g_noalloc_scratch[2 * kNoallocMaxPixels];

constexpr int kNoallocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static float4* g_noalloc_addr[kNoallocMaxDevices];

// Device address of g_noalloc_scratch on the current device (the host-side
// symbol is only a stand-in).  Looked up once per device, on the first call,
// and valid for the life of that device's context: a cudaDeviceReset unloads
// the module, after which the cached address is stale.
static dhr_status noalloc_scratch(float4** out) {
    int dev = -1;
    DHR_CUDA_TRY(cudaGetDevice(&dev));
    DHR_CHECK_ARG(dev >= 0 && dev < kNoallocMaxDevices, "svgf_atrous_noalloc: device ordinal %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        DHR_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = static_cast<float4*>(p);
    }
    *out = g_noalloc_addr[dev];
    return DHR_OK;
}

template <dhr_precision P>
static dhr_status run_atrous_noalloc(const dhr_gbuffer* g, const float4* illum, const dhr_svgf_params* prm,
                                     float* ao_out, float* sh_out, float4* scratch, cudaStream_t st) {
    const SvgfConsts k = make_consts(g->width, g->height, prm);
    const int nsq = atrous_nsq(prm);
    const auto* gd = static_cast<const typename Store<P>::G*>(g->depth_normal);
    const int L = (int)prm->levels;
    const float4* in = illum;
    for (int l = 0; l < L; ++l) {
        float4* out = scratch + (size_t)(l & 1) * kNoallocMaxPixels;
        DHR_TRY(launch_atrous<P>(l == L - 1 ? 2 : 0, nsq, atrous_radius(prm), st, k, 1 << l, gd, in, out, nullptr,
                                 ao_out, sh_out));
        in = out;
    }
    return DHR_OK;
}

}  // namespace dhr

extern "C" dhr_status dhr_svgf_atrous_noalloc(const dhr_gbuffer* gbuf, const float* illum,
                                              const dhr_svgf_params* params, float* ao_out, float* shadow_out,
                                              void* stream) {
    clear_error();
    DHR_CHECK_ARG(gbuf && gbuf->depth_normal && illum && params && ao_out && shadow_out,
                  "svgf_atrous_noalloc: null pointer");
    DHR_CHECK_ARG(gbuf->width > 0 && gbuf->height > 0, "svgf_atrous_noalloc: bad size %dx%d", gbuf->width,
                  gbuf->height);
    DHR_CHECK_ARG((int64_t)gbuf->width * gbuf->height <= kNoallocMaxPixels,
                  "svgf_atrous_noalloc: %dx%d = %lld pixels exceeds the fixed scratch of %lld pixels",
                  gbuf->width, gbuf->height, (long long)gbuf->width * gbuf->height,
                  (long long)kNoallocMaxPixels);
    DHR_CHECK_ARG(gbuf->precision == DHR_FP32 || gbuf->precision == DHR_FP16, "svgf_atrous_noalloc: bad precision");
    DHR_CHECK_ARG(((uintptr_t)illum & 15) == 0 && ((uintptr_t)gbuf->depth_normal & 15) == 0,
                  "svgf_atrous_noalloc: illum and the G-buffer must be 16-byte aligned");
    DHR_TRY(check_svgf_params(params));
    DHR_CHECK_ARG(params->levels >= 1, "svgf_atrous_noalloc: levels must be in 1..8");
    float4* scratch = nullptr;
    DHR_TRY(noalloc_scratch(&scratch));
    const float4* in = reinterpret_cast<const float4*>(illum);
    if (gbuf->precision == DHR_FP16)
        return run_atrous_noalloc<DHR_FP16>(gbuf, in, params, ao_out, shadow_out, scratch, as_stream(stream));
    return run_atrous_noalloc<DHR_FP32>(gbuf, in, params, ao_out, shadow_out, scratch, as_stream(stream));
}
