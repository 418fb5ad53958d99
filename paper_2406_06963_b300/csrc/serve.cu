// Serving form: many thin-client sessions on one GPU with continuous
// batching.
//
// The paper serves each client from a remote server (Section 1, Section 4);
// this is the B300 way of serving many of them at once.  A session is a
// client stream at its own resolution with its own SVGF history on the
// device; it is admitted only if its buffers fit the server's device-memory
// budget.  Requests (a camera pose to trace, optionally the pose to warp the
// result to -- the delay reprojection of Section 4.1) queue on the host; a
// session's newer request replaces an older one that has not started
// (latest wins, the older one is reported as dropped).  Each batch takes at
// most one request per session that has no frame in flight, writes a small
// work table into pinned memory, and replays a CUDA graph captured once per
// batch slot: the table's host-to-device copy, then persistent kernels that
// walk the tiles of every session in the batch (trace, temporal, a-trous x
// levels, target G-buffer, delay warp).  Two slots on two streams let the
// next batch be staged and launched while the previous one runs.
#include <algorithm>
#include <chrono>
#include <deque>
#include <vector>

#include "svgf_kernels.cuh"
#include "trace_device.cuh"

namespace dhr {
namespace {

constexpr int kMaxItems = 64;
// default pixel cap of one batch, about one 1920x1080 frame: under overload
// a request then waits behind ~2 ms of work instead of a whole round of
// sessions (measured on the 32-client workload: p50 52 -> 13 ms, p99 86 ->
// 37 ms at the same pixel throughput)
constexpr uint64_t kDefaultBatchPx = 2u << 20;
constexpr int kTileW = 32, kTileH = 8;

struct ServeItem {
    TraceConsts tk;          // traced pose and trace parameters
    TraceConsts tk_target;   // pose to warp to (primary rays only)
    dhr_camera cam_prev;     // previous traced pose of the session
    SvgfConsts sk;
    int has_prev, warp;
    int tile_begin, tiles_x;
    float4* g_cur;
    uint32_t* m_cur;
    const float4* g_prev;
    const uint32_t* m_prev;
    uint8_t* mask;
    uint8_t* ao;
    float2* col;
    const float4* mom_in;
    const uint8_t* hist_in;
    float4* mom_out;
    uint8_t* hist_out;
    float4* illum;
    float4* pp[2];
    float* out_ao;
    float* out_sh;
    float4* g_tgt;
    uint32_t* m_tgt;
    float* fin_ao;
    float* fin_sh;
};

struct BatchTable {
    int n_items;
    int n_tiles;
    int levels;
    int nsq;
    ServeItem items[kMaxItems];
};

__device__ __forceinline__ int find_item(const BatchTable& b, int t) {
    int lo = 0, hi = b.n_items - 1;
    while (lo < hi) {            // last item with tile_begin <= t
        const int mid = (lo + hi + 1) >> 1;
        if (b.items[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int2 tile_origin(const ServeItem& it, int t) {
    const int local = t - it.tile_begin;
    return make_int2((local % it.tiles_x) * kTileW, (local / it.tiles_x) * kTileH);
}

// each warp of the 256-thread block takes an 8x4 piece of the 32x8 tile
__device__ __forceinline__ int2 trace_thread_pixel(int2 o) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    return make_int2(o.x + (warp & 3) * 8 + (lane & 7), o.y + (warp >> 2) * 4 + (lane >> 3));
}

__global__ void __launch_bounds__(256) serve_trace_kernel(SceneView sc, const BatchTable* tb, int primary_target) {
    const BatchTable& b = *tb;
    for (int t = blockIdx.x; t < b.n_tiles; t += gridDim.x) {
        const ServeItem& it = b.items[find_item(b, t)];
        const int2 px = trace_thread_pixel(tile_origin(it, t));
        if (primary_target) {
            if (it.warp)
                trace_pixel<false, false, true>(sc, it.tk_target, px, it.g_tgt, it.m_tgt, nullptr, nullptr, nullptr);
        } else {
            trace_pixel<false, false, false>(sc, it.tk, px, it.g_cur, it.m_cur, it.mask, it.ao, nullptr);
        }
    }
}

__global__ void __launch_bounds__(256) serve_temporal_kernel(const BatchTable* tb) {
    const BatchTable& b = *tb;
    for (int t = blockIdx.x; t < b.n_tiles; t += gridDim.x) {
        const ServeItem& it = b.items[find_item(b, t)];
        const int2 o = tile_origin(it, t);
        temporal_tile<DHR_FP32, SigCounts>(it.sk, it.tk.cam, it.has_prev ? it.cam_prev : it.tk.cam, it.g_cur,
                                           it.m_cur, it.has_prev ? it.g_prev : nullptr,
                                           it.has_prev ? it.m_prev : nullptr,
                                           SigCounts{it.mask, it.ao, it.sk.inv_spp, it.sk.shadow_bit}, it.col, it.mom_in, it.hist_in,
                                           it.mom_out, it.hist_out, it.illum, o.x, o.y);
    }
}

template <int kMode, int kNsq, int kR>
__device__ __forceinline__ void serve_atrous_tile(const ServeItem& it, int l, int t, AtrousSmem& sm) {
    const float4* in = l == 0 ? it.illum : it.pp[(l - 1) & 1];
    atrous_tile<DHR_FP32, kMode, kNsq, kR>(it.sk, 1 << l, t - it.tile_begin, it.g_cur, in, it.pp[l & 1], it.col,
                                           it.out_ao, it.out_sh, sm);
}

// level l of every session; mode: 1 writes the colour history, 2 the outputs.
// The session's a-trous tiles are its 32x8 pixel tiles.
template <int kNsq, int kR>
__global__ void __launch_bounds__(256) serve_atrous_kernel(const BatchTable* tb, int l, int mode) {
    __shared__ AtrousSmem sm;
    const BatchTable& b = *tb;
    for (int t = blockIdx.x; t < b.n_tiles; t += gridDim.x) {
        const ServeItem& it = b.items[find_item(b, t)];
        if (mode == 2) serve_atrous_tile<2, kNsq, kR>(it, l, t, sm);
        else if (mode == 1) serve_atrous_tile<1, kNsq, kR>(it, l, t, sm);
        else serve_atrous_tile<0, kNsq, kR>(it, l, t, sm);
    }
}

// single-level sessions: the level-0 output is both history and result
__global__ void __launch_bounds__(256) serve_copy_kernel(const BatchTable* tb) {
    const BatchTable& b = *tb;
    for (int t = blockIdx.x; t < b.n_tiles; t += gridDim.x) {
        const ServeItem& it = b.items[find_item(b, t)];
        const int2 o = tile_origin(it, t);
        const int x = o.x + threadIdx.x, y = o.y + threadIdx.y;
        if (x >= it.sk.W || y >= it.sk.H) continue;
        const int p = y * it.sk.W + x;
        const float4 v = b.levels == 0 ? it.illum[p] : it.pp[0][p];
        it.col[p] = make_float2(v.x, v.y);
        it.out_ao[p] = v.x;
        it.out_sh[p] = v.y;
    }
}

// Delay reprojection: each pixel of the target pose's G-buffer takes the
// filtered value of the nearest valid pixel of the traced pose (the
// history-tap validity rule of the temporal step; nearest = largest bilinear
// weight among the valid taps, ties to the first); without a valid tap it
// gets 1 (no ray-traced occlusion: the client's plain local rendering).
__device__ __forceinline__ void warp_pixel(int x, int y, int W, int H, const dhr_camera& cam_tgt,
                                           const dhr_camera& cam_src, const float4* g_tgt, const uint32_t* m_tgt,
                                           const float4* g_src, const uint32_t* m_src, const float* src_ao,
                                           const float* src_sh, float* out_ao, float* out_sh) {
    using S = Store<DHR_FP32>;
    const int p = y * W + x;
    const float4 zt = g_tgt[p];
    float ao = 1.f, sh = 1.f;
    if (is_fg(zt.x)) {
        const float2 gz = depth_grad<S>(g_tgt, W, H, x, y, zt.x);
        Reproj r;
        if (reproject<S>(cam_tgt, cam_src, W, H, x, y, zt, m_tgt[p], fmaxf(fabsf(gz.x), fabsf(gz.y)), g_src, m_src,
                         r)) {
            int best = -1;
            float bw = -1.f;
            for (int k = 0; k < 4; ++k)
                if ((r.ok & (1 << k)) && r.w[k] > bw) {
                    bw = r.w[k];
                    best = k;
                }
            const int q = (r.y0 + (best >> 1)) * W + (r.x0 + (best & 1));
            ao = src_ao[q];
            sh = src_sh[q];
        }
    }
    out_ao[p] = ao;
    out_sh[p] = sh;
}

__global__ void __launch_bounds__(256) serve_warp_kernel(const BatchTable* tb) {
    const BatchTable& b = *tb;
    for (int t = blockIdx.x; t < b.n_tiles; t += gridDim.x) {
        const ServeItem& it = b.items[find_item(b, t)];
        const int2 o = tile_origin(it, t);
        const int x = o.x + threadIdx.x, y = o.y + threadIdx.y;
        const int W = it.sk.W, H = it.sk.H;
        if (x >= W || y >= H) continue;
        if (!it.warp) {
            const int p = y * W + x;
            it.fin_ao[p] = it.out_ao[p];
            it.fin_sh[p] = it.out_sh[p];
            continue;
        }
        warp_pixel(x, y, W, H, it.tk_target.cam, it.tk.cam, it.g_tgt, it.m_tgt, it.g_cur, it.m_cur, it.out_ao,
                   it.out_sh, it.fin_ao, it.fin_sh);
    }
}

__global__ void __launch_bounds__(256) warp_kernel(int W, int H, dhr_camera cam_tgt, dhr_camera cam_src,
                                                   const float4* g_tgt, const uint32_t* m_tgt, const float4* g_src,
                                                   const uint32_t* m_src, const float* src_ao, const float* src_sh,
                                                   float* out_ao, float* out_sh) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= H) return;
    warp_pixel(x, y, W, H, cam_tgt, cam_src, g_tgt, m_tgt, g_src, m_src, src_ao, src_sh, out_ao, out_sh);
}

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace
}  // namespace dhr

using namespace dhr;

namespace {

struct Request {
    uint64_t id = 0;
    int session = -1;
    dhr_camera cam{}, cam_target{};
    bool warp = false;
    uint32_t frame = 0;
    uint64_t t_arrival = 0;
};

struct Session {
    bool open = false;
    int w = 0, h = 0;
    uint64_t bytes = 0;
    void* mem = nullptr;       // one allocation for all buffers
    float4* g[2] = {nullptr, nullptr};
    uint32_t* m[2] = {nullptr, nullptr};
    uint8_t* mask = nullptr;
    uint8_t* ao = nullptr;
    float2* col = nullptr;
    float4* mom[2] = {nullptr, nullptr};
    uint8_t* hist[2] = {nullptr, nullptr};
    float4* illum = nullptr;
    float4* pp[2] = {nullptr, nullptr};
    float* out_ao = nullptr;
    float* out_sh = nullptr;
    float4* g_tgt = nullptr;
    uint32_t* m_tgt = nullptr;
    float* fin_ao = nullptr;
    float* fin_sh = nullptr;
    dhr_camera cam_prev{};
    bool has_prev = false;
    int cur = 0;               // index of the G-buffer / moments written last
    bool in_flight = false;
    bool pending = false;
    Request req;
    bool closing = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    BatchTable* h_table = nullptr;   // pinned
    BatchTable* d_table = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool in_flight = false;
    std::vector<Request> reqs;
    uint64_t t_launch = 0;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// byte layout of a session's buffers (offsets into one allocation)
struct Layout {
    size_t g[2], m[2], mask, ao, col, mom[2], hist[2], illum, pp[2], out_ao, out_sh, g_tgt, m_tgt, fin_ao, fin_sh, total;
};

Layout layout(int w, int h) {
    const size_t n = (size_t)w * h;
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    for (int i = 0; i < 2; ++i) {
        L.g[i] = take(n * 16);
        L.m[i] = take(n * 4);
        L.mom[i] = take(n * 16);
        L.hist[i] = take(n);
        L.pp[i] = take(n * 16);
    }
    L.mask = take(n);
    L.ao = take(n);
    L.col = take(n * 8);
    L.illum = take(n * 16);
    L.out_ao = take(n * 4);
    L.out_sh = take(n * 4);
    L.g_tgt = take(n * 16);
    L.m_tgt = take(n * 4);
    L.fin_ao = take(n * 4);
    L.fin_sh = take(n * 4);
    L.total = o;
    return L;
}

}  // namespace

struct dhr_server {
    const dhr_scene* scene = nullptr;
    uint64_t budget = 0, used = 0;
    dhr_trace_params tp{};
    dhr_svgf_params sp{};
    std::vector<Session> sessions;
    std::deque<int> order;             // sessions with pending requests, oldest first
    Slot slots[2];
    int grid_trace = 0, grid_px = 0;
    cudaEvent_t ref = nullptr;         // host time of `ref` = ref_host
    uint64_t ref_host = 0;
    std::vector<dhr_completion> done;  // finished or dropped, not yet polled
    uint64_t n_dropped = 0, n_batches = 0, n_frames = 0;
    uint64_t max_batch_px = kDefaultBatchPx;   // pixel cap of one batch (0: none)
};

static dhr_status capture_slot(dhr_server* s, Slot& sl) {
    cudaStream_t st = sl.stream;
    cudaGraph_t g = nullptr;
    DHR_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(sl.d_table, sl.h_table, sizeof(BatchTable), cudaMemcpyHostToDevice, st);
    const SceneView sv = s->scene->view();
    serve_trace_kernel<<<s->grid_trace, 256, 0, st>>>(sv, sl.d_table, 0);
    serve_temporal_kernel<<<s->grid_px, dim3(32, 8), 0, st>>>(sl.d_table);
    const int L = (int)s->sp.levels;
    const int nsq = s->sp.sigma_n == 128.0f ? 7 : -1;
    for (int l = 0; l < L; ++l) {
        const int mode = (l == L - 1 && L > 1) ? 2 : (l == 0 ? 1 : 0);
        const bool small = atrous_radius(&s->sp) == 1;
        if (nsq == 7 && !small) serve_atrous_kernel<7, 2><<<s->grid_px, dim3(32, 8), 0, st>>>(sl.d_table, l, mode);
        else if (!small) serve_atrous_kernel<-1, 2><<<s->grid_px, dim3(32, 8), 0, st>>>(sl.d_table, l, mode);
        else if (nsq == 7) serve_atrous_kernel<7, 1><<<s->grid_px, dim3(32, 8), 0, st>>>(sl.d_table, l, mode);
        else serve_atrous_kernel<-1, 1><<<s->grid_px, dim3(32, 8), 0, st>>>(sl.d_table, l, mode);
    }
    if (L <= 1) serve_copy_kernel<<<s->grid_px, dim3(32, 8), 0, st>>>(sl.d_table);
    serve_trace_kernel<<<s->grid_trace, 256, 0, st>>>(sv, sl.d_table, 1);
    serve_warp_kernel<<<s->grid_px, dim3(32, 8), 0, st>>>(sl.d_table);
    const cudaError_t e_launch = cudaGetLastError();
    const cudaError_t e_end = cudaStreamEndCapture(st, &g);
    if (e_launch != cudaSuccess || e_end != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return set_error(DHR_ERR_CUDA, "server: graph capture failed: %s",
                         cudaGetErrorString(e_launch != cudaSuccess ? e_launch : e_end));
    }
    const cudaError_t e = cudaGraphInstantiate(&sl.graph, g, 0);
    cudaGraphDestroy(g);
    DHR_CUDA_TRY(e);
    return DHR_OK;
}

extern "C" uint64_t dhr_server_now_ns(void) { return now_ns(); }

extern "C" dhr_status dhr_delay_warp(const dhr_gbuffer* target, const dhr_camera* cam_target, const dhr_gbuffer* source,
                                     const dhr_camera* cam_source, const float* src_ao, const float* src_shadow,
                                     float* out_ao, float* out_shadow, void* stream) {
    clear_error();
    DHR_CHECK_ARG(target && cam_target && source && cam_source && src_ao && src_shadow && out_ao && out_shadow,
                  "delay_warp: null pointer");
    DHR_CHECK_ARG(target->precision == DHR_FP32 && source->precision == DHR_FP32, "delay_warp: FP32 G-buffers only");
    const int W = target->width, H = target->height;
    DHR_CHECK_ARG(W > 0 && H > 0 && source->width == W && source->height == H && cam_target->width == W &&
                      cam_target->height == H && cam_source->width == W && cam_source->height == H,
                  "delay_warp: size mismatch");
    const dim3 grid((W + 31) / 32, (H + 7) / 8);
    warp_kernel<<<grid, dim3(32, 8), 0, as_stream(stream)>>>(
        W, H, *cam_target, *cam_source, static_cast<const float4*>(target->depth_normal), target->mesh_id,
        static_cast<const float4*>(source->depth_normal), source->mesh_id, src_ao, src_shadow, out_ao, out_shadow);
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}

extern "C" uint64_t dhr_server_session_bytes(int32_t width, int32_t height) {
    if (width <= 0 || height <= 0) return 0;
    return layout(width, height).total;
}

extern "C" void dhr_server_destroy(dhr_server* s) {
    if (!s) return;
    for (auto& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.graph) cudaGraphExecDestroy(sl.graph);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFreeHost(sl.h_table);
        cudaFree(sl.d_table);
    }
    for (auto& se : s->sessions) cudaFree(se.mem);
    if (s->ref) cudaEventDestroy(s->ref);
    delete s;
}

extern "C" dhr_status dhr_server_create(const dhr_scene* scene, uint64_t budget_bytes, const dhr_trace_params* trace,
                                        const dhr_svgf_params* svgf, dhr_server** out) {
    clear_error();
    DHR_CHECK_ARG(scene && out, "server_create: null pointer");
    DHR_TRY(check_trace_params(trace));
    DHR_TRY(check_svgf_params(svgf));
    *out = nullptr;
    auto* s = new dhr_server();
    s->scene = scene;
    s->budget = budget_bytes;
    s->tp = *trace;
    s->sp = *svgf;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s->grid_trace = sms * 4;
    s->grid_px = sms * 8;
    dhr_status st = DHR_OK;
    for (auto& sl : s->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (!e) e = cudaEventCreateWithFlags(&sl.done, cudaEventDefault);
        if (!e) e = cudaMallocHost((void**)&sl.h_table, sizeof(BatchTable));
        if (!e) e = cudaMalloc((void**)&sl.d_table, sizeof(BatchTable));
        if (e) {
            st = set_error(DHR_ERR_CUDA, "server_create: %s", cudaGetErrorString(e));
            break;
        }
        memset(sl.h_table, 0, sizeof(BatchTable));
        st = capture_slot(s, sl);
        if (st != DHR_OK) break;
    }
    if (st == DHR_OK) {
        cudaError_t e = cudaEventCreate(&s->ref);
        if (!e) e = cudaEventRecord(s->ref, s->slots[0].stream);
        if (!e) e = cudaEventSynchronize(s->ref);
        if (e) st = set_error(DHR_ERR_CUDA, "server_create: %s", cudaGetErrorString(e));
        s->ref_host = now_ns();
    }
    if (st != DHR_OK) {
        dhr_server_destroy(s);
        return st;
    }
    *out = s;
    return DHR_OK;
}

extern "C" dhr_status dhr_server_open(dhr_server* s, int32_t width, int32_t height, int32_t* session_out) {
    clear_error();
    DHR_CHECK_ARG(s && session_out, "server_open: null pointer");
    DHR_CHECK_ARG(width > 0 && height > 0 && width <= 16384 && height <= 16384, "server_open: bad size");
    const Layout L = layout(width, height);
    if (s->used + L.total > s->budget)
        return set_error(DHR_ERR_ADMISSION, "server_open: %dx%d needs %llu bytes, %llu of %llu in use", width,
                         height, (unsigned long long)L.total, (unsigned long long)s->used,
                         (unsigned long long)s->budget);
    int id = -1;
    for (size_t i = 0; i < s->sessions.size(); ++i)
        if (!s->sessions[i].open && !s->sessions[i].in_flight && !s->sessions[i].mem) {
            id = (int)i;
            break;
        }
    if (id < 0) {
        if (s->sessions.size() >= 4096) return set_error(DHR_ERR_ADMISSION, "server_open: too many sessions");
        s->sessions.emplace_back();
        id = (int)s->sessions.size() - 1;
    }
    Session& se = s->sessions[id];
    se = Session();
    char* base = nullptr;
    DHR_CUDA_TRY(cudaMalloc((void**)&base, L.total));
    DHR_CUDA_TRY(cudaMemset(base, 0, L.total));
    se.mem = base;
    se.open = true;
    se.w = width;
    se.h = height;
    se.bytes = L.total;
    for (int i = 0; i < 2; ++i) {
        se.g[i] = reinterpret_cast<float4*>(base + L.g[i]);
        se.m[i] = reinterpret_cast<uint32_t*>(base + L.m[i]);
        se.mom[i] = reinterpret_cast<float4*>(base + L.mom[i]);
        se.hist[i] = reinterpret_cast<uint8_t*>(base + L.hist[i]);
        se.pp[i] = reinterpret_cast<float4*>(base + L.pp[i]);
    }
    se.mask = reinterpret_cast<uint8_t*>(base + L.mask);
    se.ao = reinterpret_cast<uint8_t*>(base + L.ao);
    se.col = reinterpret_cast<float2*>(base + L.col);
    se.illum = reinterpret_cast<float4*>(base + L.illum);
    se.out_ao = reinterpret_cast<float*>(base + L.out_ao);
    se.out_sh = reinterpret_cast<float*>(base + L.out_sh);
    se.g_tgt = reinterpret_cast<float4*>(base + L.g_tgt);
    se.m_tgt = reinterpret_cast<uint32_t*>(base + L.m_tgt);
    se.fin_ao = reinterpret_cast<float*>(base + L.fin_ao);
    se.fin_sh = reinterpret_cast<float*>(base + L.fin_sh);
    s->used += L.total;
    *session_out = id;
    return DHR_OK;
}

static void release_session(dhr_server* s, int id) {
    Session& se = s->sessions[id];
    cudaFree(se.mem);
    s->used -= se.bytes;
    se = Session();
}

extern "C" dhr_status dhr_server_close(dhr_server* s, int32_t id) {
    clear_error();
    DHR_CHECK_ARG(s && id >= 0 && id < (int)s->sessions.size() && s->sessions[id].open, "server_close: bad session");
    Session& se = s->sessions[id];
    if (se.pending) {
        dhr_completion c{};
        c.request_id = se.req.id;
        c.session = id;
        c.frame = se.req.frame;
        c.t_arrival_ns = se.req.t_arrival;
        c.t_done_ns = now_ns();
        c.dropped = 1;
        s->done.push_back(c);
        se.pending = false;
    }
    se.open = false;
    if (se.in_flight) se.closing = true;   // freed when its batch completes
    else release_session(s, id);
    return DHR_OK;
}

extern "C" dhr_status dhr_server_submit(dhr_server* s, int32_t id, const dhr_camera* cam,
                                        const dhr_camera* cam_target, uint32_t frame, uint64_t t_arrival_ns,
                                        uint64_t request_id) {
    clear_error();
    DHR_CHECK_ARG(s && cam, "server_submit: null pointer");
    DHR_CHECK_ARG(id >= 0 && id < (int)s->sessions.size() && s->sessions[id].open, "server_submit: bad session");
    Session& se = s->sessions[id];
    DHR_CHECK_ARG(cam->width == se.w && cam->height == se.h &&
                      (!cam_target || (cam_target->width == se.w && cam_target->height == se.h)),
                  "server_submit: camera size does not match the session");
    if (se.pending) {   // latest wins: the older request never starts
        dhr_completion c{};
        c.request_id = se.req.id;
        c.session = id;
        c.frame = se.req.frame;
        c.t_arrival_ns = se.req.t_arrival;
        c.t_done_ns = now_ns();
        c.dropped = 1;
        s->done.push_back(c);
        ++s->n_dropped;
    } else {
        s->order.push_back(id);
    }
    se.pending = true;
    se.req.id = request_id;
    se.req.session = id;
    se.req.cam = *cam;
    se.req.warp = cam_target != nullptr;
    se.req.cam_target = cam_target ? *cam_target : *cam;
    se.req.frame = frame;
    se.req.t_arrival = t_arrival_ns;
    return DHR_OK;
}

static dhr_status complete_slot(dhr_server* s, Slot& sl) {
    float ms = 0.f;
    DHR_CUDA_TRY(cudaEventElapsedTime(&ms, s->ref, sl.done));
    const uint64_t t_done = s->ref_host + (uint64_t)((double)ms * 1e6);
    for (const Request& r : sl.reqs) {
        dhr_completion c{};
        c.request_id = r.id;
        c.session = r.session;
        c.frame = r.frame;
        c.t_arrival_ns = r.t_arrival;
        c.t_start_ns = sl.t_launch;
        c.t_done_ns = t_done;
        c.batch_size = (uint32_t)sl.reqs.size();
        s->done.push_back(c);
        Session& se = s->sessions[r.session];
        se.in_flight = false;
        if (se.closing) release_session(s, r.session);
        ++s->n_frames;
    }
    sl.reqs.clear();
    sl.in_flight = false;
    return DHR_OK;
}

// collect finished batches without blocking
static dhr_status reap(dhr_server* s, bool block_one) {
    for (auto& sl : s->slots) {
        if (!sl.in_flight) continue;
        cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        DHR_CUDA_TRY(e);
        DHR_TRY(complete_slot(s, sl));
        block_one = false;
    }
    if (block_one) {
        // wait for the oldest batch in flight
        Slot* oldest = nullptr;
        for (auto& sl : s->slots)
            if (sl.in_flight && (!oldest || sl.t_launch < oldest->t_launch)) oldest = &sl;
        if (oldest) {
            DHR_CUDA_TRY(cudaEventSynchronize(oldest->done));
            DHR_TRY(complete_slot(s, *oldest));
        }
    }
    return DHR_OK;
}

extern "C" dhr_status dhr_server_set_max_batch_pixels(dhr_server* s, uint64_t max_pixels) {
    clear_error();
    DHR_CHECK_ARG(s, "server_set_max_batch_pixels: null server");
    s->max_batch_px = max_pixels;
    return DHR_OK;
}

extern "C" dhr_status dhr_server_pump(dhr_server* s, int32_t* launched) {
    clear_error();
    DHR_CHECK_ARG(s, "server_pump: null server");
    if (launched) *launched = 0;
    DHR_TRY(reap(s, false));
    Slot* sl = nullptr;
    for (auto& c : s->slots)
        if (!c.in_flight) {
            sl = &c;
            break;
        }
    if (!sl || s->order.empty()) return DHR_OK;
    BatchTable& b = *sl->h_table;
    b.n_items = 0;
    b.n_tiles = 0;
    b.levels = (int)s->sp.levels;
    b.nsq = s->sp.sigma_n == 128.0f ? 7 : -1;
    const SvgfConsts k0 = make_consts(1, 1, &s->sp);
    std::deque<int> keep;
    uint64_t batch_px = 0;
    while (!s->order.empty()) {
        const int id = s->order.front();
        s->order.pop_front();
        Session& se = s->sessions[id];
        if (!se.open || !se.pending) continue;
        const uint64_t px = (uint64_t)se.w * se.h;
        const bool full = b.n_items == kMaxItems ||
                          (s->max_batch_px && b.n_items > 0 && batch_px + px > s->max_batch_px);
        if (se.in_flight || full) {   // waits for the next batch
            keep.push_back(id);
            continue;
        }
        batch_px += px;
        const Request& r = se.req;
        ServeItem& it = b.items[b.n_items];
        it = ServeItem();
        dhr_trace_params tp = s->tp;
        tp.frame = r.frame;
        it.tk = make_trace_consts(r.cam, tp);
        it.tk_target = make_trace_consts(r.cam_target, tp);
        it.cam_prev = se.cam_prev;
        it.sk = k0;
        it.sk.W = se.w;
        it.sk.H = se.h;
        it.has_prev = se.has_prev ? 1 : 0;
        it.warp = r.warp ? 1 : 0;
        it.tiles_x = (se.w + kTileW - 1) / kTileW;
        it.tile_begin = b.n_tiles;
        b.n_tiles += it.tiles_x * ((se.h + kTileH - 1) / kTileH);
        const int cur = se.cur ^ 1, prev = se.cur;
        it.g_cur = se.g[cur];
        it.m_cur = se.m[cur];
        it.g_prev = se.g[prev];
        it.m_prev = se.m[prev];
        it.mask = se.mask;
        it.ao = se.ao;
        it.col = se.col;
        it.mom_in = se.mom[prev];
        it.hist_in = se.hist[prev];
        it.mom_out = se.mom[cur];
        it.hist_out = se.hist[cur];
        it.illum = se.illum;
        it.pp[0] = se.pp[0];
        it.pp[1] = se.pp[1];
        it.out_ao = se.out_ao;
        it.out_sh = se.out_sh;
        it.g_tgt = se.g_tgt;
        it.m_tgt = se.m_tgt;
        it.fin_ao = se.fin_ao;
        it.fin_sh = se.fin_sh;
        ++b.n_items;
        se.cur = cur;
        se.cam_prev = r.cam;
        se.has_prev = true;
        se.in_flight = true;
        se.pending = false;
        sl->reqs.push_back(r);
    }
    s->order = keep;
    if (b.n_items == 0) return DHR_OK;
    sl->t_launch = now_ns();
    DHR_CUDA_TRY(cudaGraphLaunch(sl->graph, sl->stream));
    DHR_CUDA_TRY(cudaEventRecord(sl->done, sl->stream));
    sl->in_flight = true;
    ++s->n_batches;
    if (launched) *launched = b.n_items;
    return DHR_OK;
}

extern "C" dhr_status dhr_server_poll(dhr_server* s, dhr_completion* out, int32_t max, int32_t* n_out, int32_t wait) {
    clear_error();
    DHR_CHECK_ARG(s && n_out && (max == 0 || out), "server_poll: null pointer");
    *n_out = 0;
    DHR_TRY(reap(s, wait != 0 && s->done.empty()));
    const int n = std::min<int>(max, (int)s->done.size());
    for (int i = 0; i < n; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + n);
    *n_out = n;
    return DHR_OK;
}

extern "C" dhr_status dhr_server_output(dhr_server* s, int32_t id, float** ao, float** shadow) {
    clear_error();
    DHR_CHECK_ARG(s && id >= 0 && id < (int)s->sessions.size() && s->sessions[id].open, "server_output: bad session");
    if (ao) *ao = s->sessions[id].fin_ao;
    if (shadow) *shadow = s->sessions[id].fin_sh;
    return DHR_OK;
}

extern "C" dhr_status dhr_server_get_stats(dhr_server* s, dhr_server_stats* out) {
    clear_error();
    DHR_CHECK_ARG(s && out, "server_get_stats: null pointer");
    out->budget_bytes = s->budget;
    out->used_bytes = s->used;
    int open = 0;
    for (auto& se : s->sessions) open += se.open ? 1 : 0;
    out->open_sessions = open;
    out->batches = s->n_batches;
    out->frames = s->n_frames;
    out->dropped = s->n_dropped;
    return DHR_OK;
}
