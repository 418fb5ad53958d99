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
#include <array>
#include <chrono>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "raster_device.cuh"
#include "svgf_kernels.cuh"

namespace dhr {
namespace {

constexpr int kMaxItems = 64;
// default pixel cap of one batch, about one 1920x1080 frame: under overload
// a request then waits behind ~2 ms of work instead of a whole round of
// sessions (measured on the 32-client workload: p50 52 -> 13 ms, p99 86 ->
// 37 ms at the same pixel throughput)
constexpr uint64_t kDefaultBatchPx = 2u << 20;
constexpr int kTileW = 32, kTileH = 8;
// sessions of at least this many pixels rasterise their primary visibility
// (the binning pass costs about the same at every resolution, the traversal
// it replaces grows with the pixels: measured break-even near 1.1 Mpx)
constexpr uint64_t kDefaultRasterMinPx = 1u << 17;

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
    int raster;              // primary visibility rasterised (tile lists in g_cur, big list in m_cur)
    RasterConsts rc;
    BinLayout bl;
    int raster_tgt;          // the warp target's primary visibility rasterised (lists in g_tgt, m_tgt)
    RasterConsts rc_tgt;
    BinLayout bl_tgt;
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

// The batch's trace: AO rays start at their start cells; shadow rays start
// at the root (their start cells, at 64 registers per thread here, spilled
// the kernel's traversal state and served fewer pixels per second).
__global__ void __launch_bounds__(256, 4) serve_trace_kernel(SceneView sc, const BatchTable* tb, int primary_target) {
    const BatchTable& b = *tb;
    for (int t = blockIdx.x; t < b.n_tiles; t += gridDim.x) {
        const ServeItem& it = b.items[find_item(b, t)];
        const int2 px = trace_thread_pixel(tile_origin(it, t));
        if (primary_target) {
            if (it.warp && it.raster_tgt)
                trace_pixel<false, false, true, false, true, 8>(sc, it.tk_target, px, it.g_tgt, it.m_tgt, nullptr,
                                                                nullptr, nullptr);
            else if (it.warp)
                trace_pixel<false, false, true, false, false, 8>(sc, it.tk_target, px, it.g_tgt, it.m_tgt, nullptr,
                                                                 nullptr, nullptr);
        } else if (it.raster) {
            trace_pixel<false, false, false, false, true, 8, false>(sc, it.tk, px, it.g_cur, it.m_cur, it.mask, it.ao,
                                                                    nullptr);
        } else {
            trace_pixel<false, false, false, false, false, 8, false>(sc, it.tk, px, it.g_cur, it.m_cur, it.mask,
                                                                     it.ao, nullptr);
        }
    }
}

// rasterised primary visibility of the batch's items with raster (the
// traced pose) or raster_tgt (the warp's target pose) set: clear their tile
// counts, bin every chunk of the scene, bin the listed triangles.  Layout 0
// of an item is its traced pose's, layout 1 its target's.
__device__ __forceinline__ bool bin_layout(const ServeItem& it, int l, const RasterConsts*& rc,
                                           const BinLayout*& bl) {
    if (it.tiles_x == 0 || !(l == 0 ? it.raster : it.raster_tgt)) return false;
    rc = l == 0 ? &it.rc : &it.rc_tgt;
    bl = l == 0 ? &it.bl : &it.bl_tgt;
    return true;
}

__global__ void __launch_bounds__(256) serve_bin_clear_kernel(const BatchTable* tb, int layout) {
    const BatchTable& b = *tb;
    for (int i = 0; i < b.n_items; ++i) {
        const RasterConsts* rc;
        const BinLayout* bl;
        if (!bin_layout(b.items[i], layout, rc, bl)) continue;
        for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < bl->n_tiles; t += gridDim.x * blockDim.x)
            bin_clear(*bl, t);
    }
}

__global__ void __launch_bounds__(kChunk) serve_bin_kernel(SceneView sc, const BatchTable* tb, int layout) {
    const BatchTable& b = *tb;
    const int chunks = (sc.n_tris + kChunk - 1) / kChunk;
    for (int i = 0; i < b.n_items; ++i) {
        const RasterConsts* rc;
        const BinLayout* bl;
        if (!bin_layout(b.items[i], layout, rc, bl)) continue;
        for (int c = blockIdx.x; c < chunks; c += gridDim.x) bin_chunk(sc, *rc, *bl, c);
    }
}

__global__ void __launch_bounds__(128) serve_bin_big_kernel(SceneView sc, const BatchTable* tb, int layout) {
    const BatchTable& b = *tb;
    for (int i = 0; i < b.n_items; ++i) {
        const RasterConsts* rc;
        const BinLayout* bl;
        if (bin_layout(b.items[i], layout, rc, bl)) bin_big(sc, *rc, *bl, blockIdx.x, gridDim.x);
    }
}

__global__ void __launch_bounds__(256, 5) serve_temporal_kernel(const BatchTable* tb) {
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
__global__ void __launch_bounds__(256, 4) serve_atrous_kernel(const BatchTable* tb, int l, int mode) {
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

// ------------------------------------------------------------------------
// Device-resident request loop.  One graph launch runs a WHILE conditional
// node whose body is a scheduling kernel followed by an IF node holding the
// stages of a batch.  The host only writes requests into per-session
// mailboxes and reads completion records, both in mapped host memory; the
// loop picks requests, builds the batch table in device memory, runs the
// stages and publishes completions without returning to the host.  It ends
// when the host asks it to stop, when no request has arrived for the idle
// limit (status DHR_ERR_TIMEOUT), or at a hard limit on its run time and
// iterations; no kernel of it waits on another kernel, and the one wait it
// has (for requests, inside a scheduling pass) is bounded by %globaltimer
// and a pass count.
// ------------------------------------------------------------------------
constexpr int kLoopMaxSessions = 1024;
constexpr uint64_t kRingRecords = 1u << 14;
constexpr int kLoopPolls = 64;          // polls of the mailboxes in one scheduling pass
// loops running side by side on their own streams over the same mailboxes
// (a session is claimed by one of them at a time), so that one batch's
// tail overlaps the next batch's head, as two host-launched slots do
constexpr int kLoops = 2;

// host -> device, one per session slot; the host is the only writer.  seq
// is odd while the host writes and 2k once request k (k = 1, 2, ...) is
// complete: a newer request replaces an untaken older one (latest wins).
struct alignas(16) Mailbox {
    uint32_t seq;
    uint32_t warp;
    uint32_t frame;
    uint32_t pad;
    uint64_t t_arrival;
    uint64_t request_id;
    dhr_camera cam;
    dhr_camera cam_target;
};

// host -> device, one per session slot: its buffers.  generation is odd
// while the host writes and even when stable; a new even value is a new
// session (the loop resets its per-session state).
struct alignas(16) SessionSlot {
    uint32_t generation;
    int32_t open;
    int32_t w, h;
    float4* g[2];
    uint32_t* m[2];
    float4* mom[2];
    uint8_t* hist[2];
    float4* pp[2];
    uint8_t* mask;
    uint8_t* ao;
    float2* col;
    float4* illum;
    float* out_ao;
    float* out_sh;
    float4* g_tgt;
    uint32_t* m_tgt;
    float* fin_ao;
    float* fin_sh;
};

// loop control, mapped; each field has one writer
struct alignas(64) LoopCtl {
    uint32_t stop;              // host: 1 = end the loops
    uint32_t n_slots;           // host: session slots in use
    uint64_t max_batch_px;      // host: pixel cap of one batch (0: none)
    uint64_t ring_tail;         // host: completion records consumed
    uint64_t epoch[kLoops];     // device: scheduling passes done, per loop
    uint32_t status[kLoops];    // device: DHR_OK or DHR_ERR_TIMEOUT once ended
    uint32_t running[kLoops];   // device: 0 once that loop has ended
};

// shared by the loops (device memory)
struct LoopShared {
    unsigned long long reserve;     // ring positions handed out
    unsigned long long last_work;   // %globaltimer of the last request taken by any loop
    unsigned long long t0;          // %globaltimer when the first loop started
};

struct alignas(16) LoopRecord {   // device -> host
    uint64_t request_id;
    uint64_t t_start;         // %globaltimer when its batch was scheduled
    uint64_t t_done;          // %globaltimer when its batch completed
    int32_t session;
    uint32_t k;               // request index within the session
    uint32_t frame;
    uint32_t batch_size;
    uint32_t generation;      // of the session slot
    uint32_t pad;
    uint64_t seq;             // ring position + 1, written last
};

// per-session state kept by the loop (device memory)
struct DevSession {
    uint32_t generation;
    uint32_t taken;           // index of the last request taken
    int32_t cur;              // G-buffer / moments index written last
    int32_t has_prev;
    dhr_camera cam_prev;
    uint32_t busy;            // 1 while a loop holds the session (claimed with atomicCAS)
};

struct LoopLimits {
    uint64_t idle_ns;
    uint64_t max_run_ns;
    uint64_t poll_ns;
    uint64_t max_iters;
};

// one loop's own state (device memory)
struct LoopMeta {
    uint64_t iters;
    LoopLimits lim;
    TraceConsts tk_base;      // lights, cones, AO parameters; camera and frame per request
    SvgfConsts sk_base;
    int32_t levels, nsq;
    uint64_t raster_min_px;   // sessions of at least this many pixels rasterise (~0: none)
    int32_t n_items;
    uint64_t t_batch;
    int32_t item_session[kMaxItems];
    uint32_t item_k[kMaxItems];
    uint32_t item_frame[kMaxItems];
    uint32_t item_gen[kMaxItems];
    uint64_t item_request[kMaxItems];
};

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_acquire_sys64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys64(uint64_t* p, uint64_t v) {
    asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One scheduling pass of loop `li` (one block of 1024 threads, thread i
// looks after session slot i): end the loop if asked or past a limit; else
// wait up to poll_ns for requests of sessions no loop holds, claim one per
// session -- oldest arrival first, at most kMaxItems and the pixel cap --
// and build the batch table.
__global__ void __launch_bounds__(1024) loop_schedule_kernel(int li, LoopCtl* ctl, const Mailbox* mb,
                                                             const SessionSlot* slots, DevSession* ds,
                                                             LoopShared* sh, LoopMeta* meta, BatchTable* tb,
                                                             cudaGraphConditionalHandle h_loop,
                                                             cudaGraphConditionalHandle h_work) {
    __shared__ uint64_t key[kLoopMaxSessions];
    __shared__ uint32_t sreq[kLoopMaxSessions];
    __shared__ uint32_t sgen[kLoopMaxSessions];
    __shared__ uint64_t spx[kLoopMaxSessions];
    __shared__ int order[kLoopMaxSessions];
    __shared__ int s_end, s_count, s_go, s_n;
    __shared__ uint64_t s_now;
    const LoopLimits lim = meta->lim;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const uint64_t now = globaltimer();
        if (meta->iters == 0) {
            atomicCAS(&sh->t0, 0ull, (unsigned long long)now);
            atomicMax(&sh->last_work, (unsigned long long)now);
        }
        const uint64_t t0 = *(volatile unsigned long long*)&sh->t0;
        int end = 0;
        if (ld_acquire_sys(&ctl->stop)) end = 1;
        else if (now - t0 > lim.max_run_ns || meta->iters >= lim.max_iters) end = 2;
        s_end = end;
        s_now = now;
    }
    __syncthreads();
    const uint32_t n_slots = min(ld_acquire_sys(&ctl->n_slots), (uint32_t)kLoopMaxSessions);
    // room for both loops' completion records
    const uint64_t reserved = *(volatile unsigned long long*)&sh->reserve;
    const bool room = reserved - ld_acquire_sys64(&ctl->ring_tail) + 2 * kLoops * kMaxItems <= kRingRecords;
    int count = 0;
    if (!s_end) {
        for (int pass = 0; pass < kLoopPolls; ++pass) {
            uint64_t k = ~0ull;
            if (room && tid < (int)n_slots) {
                const SessionSlot* sl = slots + tid;
                const uint32_t g1 = ld_acquire_sys(&sl->generation);
                DevSession& d = ds[tid];
                bool fresh = !(g1 & 1u) && g1 != 0u;
                if (fresh && *(volatile uint32_t*)&d.generation != g1) {
                    // a new session in this slot: reset its state, holding it
                    if (atomicCAS(&d.busy, 0u, 1u) == 0u) {
                        d.generation = g1;
                        d.taken = 0;
                        d.cur = 0;
                        d.has_prev = 0;
                        __threadfence();
                        atomicExch(&d.busy, 0u);
                    }
                    fresh = false;
                }
                if (fresh && *(volatile uint32_t*)&d.busy == 0u) {
                    const uint32_t s1 = ld_acquire_sys(&mb[tid].seq);
                    if (!(s1 & 1u) && (s1 >> 1) > *(volatile uint32_t*)&d.taken && sl->open) {
                        const uint64_t ta = *(volatile const uint64_t*)&mb[tid].t_arrival;
                        const uint64_t px = (uint64_t)sl->w * (uint64_t)sl->h;
                        __threadfence_system();
                        if (ld_acquire_sys(&mb[tid].seq) == s1 && ld_acquire_sys(&sl->generation) == g1) {
                            k = ta;
                            sreq[tid] = s1;
                            sgen[tid] = g1;
                            spx[tid] = px;
                        }
                    }
                }
            }
            if (tid < kLoopMaxSessions) key[tid] = k;
            count = __syncthreads_count(k != ~0ull);
            if (tid == 0) s_go = count > 0 || globaltimer() - s_now > lim.poll_ns;
            __syncthreads();
            if (s_go) break;
            __nanosleep(2000);
        }
    }
    if (tid == 0) s_count = count;
    __syncthreads();
    // rank the candidates by arrival (ties: slot index)
    if (!s_end && tid < (int)n_slots && key[tid] != ~0ull) {
        const uint64_t mine = key[tid];
        int rank = 0;
        for (int j = 0; j < (int)n_slots; ++j) {
            const uint64_t kj = key[j];
            rank += (kj < mine || (kj == mine && j < tid)) ? 1 : 0;
        }
        order[rank] = tid;
    }
    __syncthreads();
    if (tid == 0) {
        int n = 0;
        if (!s_end) {
            const uint64_t cap = *(volatile const uint64_t*)&ctl->max_batch_px;
            uint64_t px = 0;
            for (int r = 0; r < s_count && n < kMaxItems; ++r) {
                const int id = order[r];
                if (cap && n > 0 && px + spx[id] > cap) break;
                px += spx[id];
                order[n++] = id;    // order[0..n) now the sessions to claim
            }
        }
        s_n = n;
    }
    __syncthreads();
    // build the items, one thread each; a session the other loop claimed
    // first, or whose request was replaced while it was read, is left out
    if (tid < s_n) {
        const int id = order[tid];
        const Mailbox& m = mb[id];
        const SessionSlot& sl = slots[id];
        DevSession& d = ds[id];
        ServeItem& it = tb->items[tid];
        it = ServeItem();
        const bool claimed = atomicCAS(&d.busy, 0u, 1u) == 0u;
        __threadfence();
        bool valid = claimed && *(volatile uint32_t*)&d.generation == sgen[id] &&
                     (sreq[id] >> 1) > *(volatile uint32_t*)&d.taken;
        dhr_camera cam, cam_t;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&m.cam);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&cam);
        for (int w = 0; w < (int)(sizeof(dhr_camera) / 4); ++w) dst[w] = ((volatile const uint32_t*)src)[w];
        src = reinterpret_cast<const uint32_t*>(&m.cam_target);
        dst = reinterpret_cast<uint32_t*>(&cam_t);
        for (int w = 0; w < (int)(sizeof(dhr_camera) / 4); ++w) dst[w] = ((volatile const uint32_t*)src)[w];
        const uint32_t frame = *(volatile const uint32_t*)&m.frame;
        const uint32_t warp = *(volatile const uint32_t*)&m.warp;
        const uint64_t rid = *(volatile const uint64_t*)&m.request_id;
        it.tk = meta->tk_base;
        it.tk.cam = cam;
        it.tk.frame = frame;
        it.tk_target = meta->tk_base;
        it.tk_target.cam = cam_t;
        it.tk_target.frame = frame;
        it.cam_prev = d.cam_prev;
        it.sk = meta->sk_base;
        it.sk.W = sl.w;
        it.sk.H = sl.h;
        it.has_prev = d.has_prev;
        it.warp = warp ? 1 : 0;
        it.tiles_x = (sl.w + kTileW - 1) / kTileW;
        const int cur = d.cur ^ 1, prev = d.cur;
        it.g_cur = sl.g[cur];
        it.m_cur = sl.m[cur];
        it.g_prev = sl.g[prev];
        it.m_prev = sl.m[prev];
        it.mask = sl.mask;
        it.ao = sl.ao;
        it.col = sl.col;
        it.mom_in = sl.mom[prev];
        it.hist_in = sl.hist[prev];
        it.mom_out = sl.mom[cur];
        it.hist_out = sl.hist[cur];
        it.illum = sl.illum;
        it.pp[0] = sl.pp[0];
        it.pp[1] = sl.pp[1];
        it.out_ao = sl.out_ao;
        it.out_sh = sl.out_sh;
        it.g_tgt = sl.g_tgt;
        it.m_tgt = sl.m_tgt;
        it.fin_ao = sl.fin_ao;
        it.fin_sh = sl.fin_sh;
        // (the tile layout follows the camera's size, which must be the session's)
        it.raster = (uint64_t)sl.w * sl.h >= meta->raster_min_px && cam.width == sl.w && cam.height == sl.h &&
                    make_raster(cam, it.g_cur, it.m_cur, 4, it.rc, it.bl);
        it.raster_tgt = warp && (uint64_t)sl.w * sl.h >= meta->raster_min_px && cam_t.width == sl.w &&
                        cam_t.height == sl.h && make_raster(cam_t, it.g_tgt, it.m_tgt, 4, it.rc_tgt, it.bl_tgt);
        __threadfence_system();
        valid = valid && ld_acquire_sys(&m.seq) == sreq[id] && ld_acquire_sys(&sl.generation) == sgen[id];
        if (valid) {
            d.cur = cur;
            d.cam_prev = cam;
            d.has_prev = 1;
            d.taken = sreq[id] >> 1;
        } else {
            // not this loop's to serve: no tile and no binning pass may touch
            // the session's buffers (the loop that claimed it is using them)
            it.tiles_x = 0;
            it.raster = 0;
            it.raster_tgt = 0;
            if (claimed) {
                __threadfence();
                atomicExch(&d.busy, 0u);
            }
        }
        meta->item_session[tid] = valid ? id : -1;
        meta->item_k[tid] = sreq[id] >> 1;
        meta->item_frame[tid] = frame;
        meta->item_gen[tid] = sgen[id];
        meta->item_request[tid] = rid;
    }
    __syncthreads();
    if (tid == 0) {
        const int n = s_n;
        int tiles = 0, live = 0;
        for (int j = 0; j < n; ++j) {
            ServeItem& it = tb->items[j];
            it.tile_begin = tiles;
            if (it.tiles_x > 0) tiles += it.tiles_x * ((it.sk.H + kTileH - 1) / kTileH);
            live += meta->item_session[j] >= 0 ? 1 : 0;
        }
        tb->n_items = n;
        tb->n_tiles = tiles;
        tb->levels = meta->levels;
        tb->nsq = meta->nsq;
        meta->n_items = n;
        meta->t_batch = s_now;
        meta->iters += 1;
        st_release_sys64(&ctl->epoch[li], meta->iters);
        if (live > 0) atomicMax(&sh->last_work, (unsigned long long)s_now);
        int end = s_end;
        const uint64_t last = *(volatile unsigned long long*)&sh->last_work;
        if (!end && live == 0 && s_count == 0 && s_now > last && s_now - last > lim.idle_ns) end = 2;
        if (end) {
            st_release_sys(&ctl->status[li], end == 1 ? (uint32_t)DHR_OK : (uint32_t)DHR_ERR_TIMEOUT);
            st_release_sys(&ctl->running[li], 0u);
        }
        cudaGraphSetConditional(h_work, (!end && live > 0) ? 1u : 0u);
        cudaGraphSetConditional(h_loop, end ? 0u : 1u);
    }
}

// completion records of the batch just run (ring positions reserved from
// the shared counter, each stamped last with its position + 1), then the
// batch's sessions are released for the next request
__global__ void loop_complete_kernel(LoopRecord* ring, DevSession* ds, LoopShared* sh, LoopMeta* meta) {
    const int n = meta->n_items;
    const uint64_t now = globaltimer();
    __shared__ int s_slot[kMaxItems];
    __shared__ unsigned long long s_base;
    if (threadIdx.x == 0) {
        int live = 0;
        for (int j = 0; j < n; ++j) {
            s_slot[j] = meta->item_session[j] >= 0 ? live : -1;
            live += meta->item_session[j] >= 0 ? 1 : 0;
        }
        s_base = live > 0 ? atomicAdd(&sh->reserve, (unsigned long long)live) : 0ull;
        for (int j = 0; j < n; ++j)
            if (s_slot[j] >= 0) s_slot[j] |= live << 16;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        if (s_slot[j] < 0) continue;
        const int pos = s_slot[j] & 0xFFFF, live = s_slot[j] >> 16;
        const uint64_t at = s_base + (uint64_t)pos;
        LoopRecord* r = ring + at % kRingRecords;
        r->request_id = meta->item_request[j];
        r->t_start = meta->t_batch;
        r->t_done = now;
        r->session = meta->item_session[j];
        r->k = meta->item_k[j];
        r->frame = meta->item_frame[j];
        r->batch_size = (uint32_t)live;
        r->generation = meta->item_gen[j];
        r->pad = 0;
        __threadfence_system();
        st_release_sys64(&r->seq, at + 1);
        DevSession& d = ds[meta->item_session[j]];
        __threadfence();
        atomicExch(&d.busy, 0u);
    }
}

// %globaltimer read once (host clock calibration)
__global__ void clock_kernel(uint64_t* out) { *out = globaltimer(); }

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

// host side of the device-resident loop
struct LoopHost {
    cudaStream_t stream[kLoops] = {};
    cudaGraphExec_t exec[kLoops] = {};
    LoopShared* d_shared = nullptr;
    LoopCtl* ctl = nullptr;               // mapped
    Mailbox* mb = nullptr;                // mapped [kLoopMaxSessions]
    SessionSlot* slots = nullptr;         // mapped [kLoopMaxSessions]
    LoopRecord* ring = nullptr;           // mapped [kRingRecords]
    uint64_t* clock = nullptr;            // mapped, one %globaltimer sample
    DevSession* d_sess = nullptr;
    LoopMeta* d_meta[kLoops] = {};
    BatchTable* d_table[kLoops] = {};
    bool active = false;                  // launched and not yet collected by loop_stop
    int64_t clock_offset = 0;             // host ns - device ns
    uint32_t generation[kLoopMaxSessions] = {};
    uint32_t published[kLoopMaxSessions] = {};        // last request index written to the mailbox
    std::map<uint32_t, Request> outstanding[kLoopMaxSessions];  // published, not yet reported
    // closed sessions: (id, every loop's epoch at the close)
    std::vector<std::pair<int, std::array<uint64_t, kLoops>>> to_release;
};

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
    uint64_t raster_min_px = kDefaultRasterMinPx;   // sessions from this size rasterise primaries
    cudaStream_t mem_stream = nullptr;  // session allocations (stream ordered)
    // a batch graph's branch for the warp targets' binning and primary
    // visibility (only used while graphs are captured; lowest priority, the
    // slots' and loops' capture streams highest)
    cudaStream_t fork_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    LoopHost loop;
};

// binning of the batch's layout 0 (traced poses) or 1 (warp targets) on `st`
static void launch_bins(const SceneView& sv, cudaStream_t st, const BatchTable* tb, int layout) {
    serve_bin_clear_kernel<<<148 * 2, 256, 0, st>>>(tb, layout);
    serve_bin_kernel<<<148 * 8, kChunk, 0, st>>>(sv, tb, layout);
    serve_bin_big_kernel<<<kBigGrid, 128, 0, st>>>(sv, tb, layout);
}

// the stages of one batch on `st`, all reading the batch table `tb`:
// binning, trace, temporal, a-trous levels, delay warp; the warp target's
// binning and primary visibility form a branch of their own (fork_st) that
// joins before the warp
static void launch_stages(const dhr_server* s, cudaStream_t st, const BatchTable* tb) {
    const SceneView sv = s->scene->view();
    cudaEventRecord(s->ev_fork, st);
    cudaStreamWaitEvent(s->fork_st, s->ev_fork, 0);
    launch_bins(sv, s->fork_st, tb, 1);
    serve_trace_kernel<<<s->grid_trace, 256, 0, s->fork_st>>>(sv, tb, 1);
    cudaEventRecord(s->ev_join, s->fork_st);
    launch_bins(sv, st, tb, 0);
    serve_trace_kernel<<<s->grid_trace, 256, 0, st>>>(sv, tb, 0);
    serve_temporal_kernel<<<s->grid_px, dim3(32, 8), 0, st>>>(tb);
    const int L = (int)s->sp.levels;
    const int nsq = s->sp.sigma_n == 128.0f ? 7 : -1;
    for (int l = 0; l < L; ++l) {
        const int mode = (l == L - 1 && L > 1) ? 2 : (l == 0 ? 1 : 0);
        const bool small = atrous_radius(&s->sp) == 1;
        if (nsq == 7 && !small) serve_atrous_kernel<7, 2><<<s->grid_px, dim3(32, 8), 0, st>>>(tb, l, mode);
        else if (!small) serve_atrous_kernel<-1, 2><<<s->grid_px, dim3(32, 8), 0, st>>>(tb, l, mode);
        else if (nsq == 7) serve_atrous_kernel<7, 1><<<s->grid_px, dim3(32, 8), 0, st>>>(tb, l, mode);
        else serve_atrous_kernel<-1, 1><<<s->grid_px, dim3(32, 8), 0, st>>>(tb, l, mode);
    }
    if (L <= 1) serve_copy_kernel<<<s->grid_px, dim3(32, 8), 0, st>>>(tb);
    cudaStreamWaitEvent(st, s->ev_join, 0);
    serve_warp_kernel<<<s->grid_px, dim3(32, 8), 0, st>>>(tb);
}

static dhr_status capture_slot(dhr_server* s, Slot& sl) {
    cudaStream_t st = sl.stream;
    cudaGraph_t g = nullptr;
    DHR_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(sl.d_table, sl.h_table, sizeof(BatchTable), cudaMemcpyHostToDevice, st);
    launch_stages(s, st, sl.d_table);
    const cudaError_t e_launch = cudaGetLastError();
    const cudaError_t e_end = cudaStreamEndCapture(st, &g);
    if (e_launch != cudaSuccess || e_end != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return set_error(DHR_ERR_CUDA, "server: graph capture failed: %s",
                         cudaGetErrorString(e_launch != cudaSuccess ? e_launch : e_end));
    }
    const cudaError_t e = cudaGraphInstantiate(&sl.graph, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    DHR_CUDA_TRY(e);
    return DHR_OK;
}

// ------------------------------------------------------- device loop host
// publishes session slot `id` (open with its buffers, or closed) for the
// loop; the mailbox restarts at request 0 for a newly opened session
static void publish_slot(dhr_server* s, int id, bool open) {
    LoopHost& L = s->loop;
    if (id >= kLoopMaxSessions || !L.slots) return;
    SessionSlot& sl = L.slots[id];
    const uint32_t g = L.generation[id] + 2u;   // even, never 0
    __atomic_store_n(&sl.generation, g - 1u, __ATOMIC_RELAXED);
    __atomic_thread_fence(__ATOMIC_RELEASE);
    if (open) {
        const Session& se = s->sessions[id];
        __atomic_store_n(&L.mb[id].seq, 0u, __ATOMIC_RELAXED);
        L.published[id] = 0;
        sl.w = se.w;
        sl.h = se.h;
        for (int i = 0; i < 2; ++i) {
            sl.g[i] = se.g[i];
            sl.m[i] = se.m[i];
            sl.mom[i] = se.mom[i];
            sl.hist[i] = se.hist[i];
            sl.pp[i] = se.pp[i];
        }
        sl.mask = se.mask;
        sl.ao = se.ao;
        sl.col = se.col;
        sl.illum = se.illum;
        sl.out_ao = se.out_ao;
        sl.out_sh = se.out_sh;
        sl.g_tgt = se.g_tgt;
        sl.m_tgt = se.m_tgt;
        sl.fin_ao = se.fin_ao;
        sl.fin_sh = se.fin_sh;
    }
    sl.open = open ? 1 : 0;
    __atomic_store_n(&sl.generation, g, __ATOMIC_RELEASE);
    L.generation[id] = g;
    uint32_t n = (uint32_t)std::min<size_t>(s->sessions.size(), (size_t)kLoopMaxSessions);
    __atomic_store_n(&L.ctl->n_slots, n, __ATOMIC_RELEASE);
}

// writes request k of session id into its mailbox (the loop takes the newest)
static void publish_request(dhr_server* s, int id, const Request& r) {
    LoopHost& L = s->loop;
    const uint32_t k = ++L.published[id];
    L.outstanding[id][k] = r;
    Mailbox& m = L.mb[id];
    __atomic_store_n(&m.seq, 2u * k - 1u, __ATOMIC_RELAXED);
    __atomic_thread_fence(__ATOMIC_RELEASE);
    m.warp = r.warp ? 1u : 0u;
    m.frame = r.frame;
    m.t_arrival = r.t_arrival;
    m.request_id = r.id;
    m.cam = r.cam;
    m.cam_target = r.cam_target;
    __atomic_store_n(&m.seq, 2u * k, __ATOMIC_RELEASE);
}

static dhr_status loop_create(dhr_server* s) {
    LoopHost& L = s->loop;
    DHR_CUDA_TRY(cudaHostAlloc((void**)&L.ctl, sizeof(LoopCtl), cudaHostAllocMapped));
    DHR_CUDA_TRY(cudaHostAlloc((void**)&L.mb, sizeof(Mailbox) * kLoopMaxSessions, cudaHostAllocMapped));
    DHR_CUDA_TRY(cudaHostAlloc((void**)&L.slots, sizeof(SessionSlot) * kLoopMaxSessions, cudaHostAllocMapped));
    DHR_CUDA_TRY(cudaHostAlloc((void**)&L.ring, sizeof(LoopRecord) * kRingRecords, cudaHostAllocMapped));
    DHR_CUDA_TRY(cudaHostAlloc((void**)&L.clock, sizeof(uint64_t), cudaHostAllocMapped));
    memset(L.ctl, 0, sizeof(LoopCtl));
    memset(L.mb, 0, sizeof(Mailbox) * kLoopMaxSessions);
    memset(L.slots, 0, sizeof(SessionSlot) * kLoopMaxSessions);
    memset(L.ring, 0, sizeof(LoopRecord) * kRingRecords);
    DHR_CUDA_TRY(cudaMalloc((void**)&L.d_sess, sizeof(DevSession) * kLoopMaxSessions));
    DHR_CUDA_TRY(cudaMalloc((void**)&L.d_shared, sizeof(LoopShared)));
    LoopCtl* ctl_d = nullptr;
    Mailbox* mb_d = nullptr;
    SessionSlot* slots_d = nullptr;
    LoopRecord* ring_d = nullptr;
    DHR_CUDA_TRY(cudaHostGetDevicePointer((void**)&ctl_d, L.ctl, 0));
    DHR_CUDA_TRY(cudaHostGetDevicePointer((void**)&mb_d, L.mb, 0));
    DHR_CUDA_TRY(cudaHostGetDevicePointer((void**)&slots_d, L.slots, 0));
    DHR_CUDA_TRY(cudaHostGetDevicePointer((void**)&ring_d, L.ring, 0));
    for (int li = 0; li < kLoops; ++li) {
        int least = 0, greatest = 0;
        DHR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        DHR_CUDA_TRY(cudaStreamCreateWithPriority(&L.stream[li], cudaStreamNonBlocking, greatest));
        DHR_CUDA_TRY(cudaMalloc((void**)&L.d_meta[li], sizeof(LoopMeta)));
        DHR_CUDA_TRY(cudaMalloc((void**)&L.d_table[li], sizeof(BatchTable)));
        DHR_CUDA_TRY(cudaMemset(L.d_table[li], 0, sizeof(BatchTable)));
        cudaStream_t st = L.stream[li];
        // WHILE (loop) { schedule; IF (work) { stages; completions } }
        cudaGraph_t g = nullptr;
        DHR_CUDA_TRY(cudaGraphCreate(&g, 0));
        cudaGraphConditionalHandle h_loop, h_work;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h_loop, g, 1u, cudaGraphCondAssignDefault);
        cudaGraphNodeParams wp = {};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = h_loop;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wnode = nullptr;
        if (!e) e = cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &wp);
        cudaGraph_t body = e ? nullptr : wp.conditional.phGraph_out[0];
        if (!e) e = cudaGraphConditionalHandleCreate(&h_work, body, 0u, 0u);
        cudaGraph_t captured = nullptr;
        if (!e) e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (!e) {
            loop_schedule_kernel<<<1, 1024, 0, st>>>(li, ctl_d, mb_d, slots_d, L.d_sess, L.d_shared, L.d_meta[li],
                                                      L.d_table[li], h_loop, h_work);
            e = cudaGetLastError();
            const cudaError_t e2 = cudaStreamEndCapture(st, &captured);
            if (!e) e = e2;
        }
        cudaGraphNode_t sched = nullptr;
        size_t n_nodes = 1;
        if (!e) e = cudaGraphGetNodes(body, &sched, &n_nodes);
        cudaGraphNodeParams ip = {};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = h_work;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t inode = nullptr;
        if (!e && n_nodes != 1) e = cudaErrorInvalidValue;
        if (!e) e = cudaGraphAddNode(&inode, body, &sched, nullptr, 1, &ip);
        if (!e) {
            cudaGraph_t ifbody = ip.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(st, ifbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (!e) {
                launch_stages(s, st, L.d_table[li]);
                loop_complete_kernel<<<1, 64, 0, st>>>(ring_d, L.d_sess, L.d_shared, L.d_meta[li]);
                e = cudaGetLastError();
                const cudaError_t e2 = cudaStreamEndCapture(st, &captured);
                if (!e) e = e2;
            }
        }
        if (!e) e = cudaGraphInstantiate(&L.exec[li], g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        if (e) return set_error(DHR_ERR_CUDA, "server: device loop graph: %s", cudaGetErrorString(e));
    }
    return DHR_OK;
}

static void loop_destroy(LoopHost& L) {
    for (int li = 0; li < kLoops; ++li) {
        if (L.exec[li]) cudaGraphExecDestroy(L.exec[li]);
        if (L.stream[li]) cudaStreamDestroy(L.stream[li]);
        cudaFree(L.d_meta[li]);
        cudaFree(L.d_table[li]);
    }
    cudaFreeHost(L.ctl);
    cudaFreeHost(L.mb);
    cudaFreeHost(L.slots);
    cudaFreeHost(L.ring);
    cudaFreeHost(L.clock);
    cudaFree(L.d_sess);
    cudaFree(L.d_shared);
}

// records written by the loop since the last call: completions, and the
// requests they superseded as dropped
static void loop_collect(dhr_server* s) {
    LoopHost& L = s->loop;
    uint64_t tail = L.ctl->ring_tail;
    uint64_t last_batch = ~0ull;
    for (;; ++tail) {
        // records are stamped with their position + 1 once written (the
        // loops fill their reserved positions in any order)
        LoopRecord* slot = L.ring + tail % kRingRecords;
        if (__atomic_load_n(&slot->seq, __ATOMIC_ACQUIRE) != tail + 1) break;
        const LoopRecord r = *slot;
        if (r.session < 0 || r.session >= kLoopMaxSessions || r.generation != L.generation[r.session]) continue;
        auto& out = L.outstanding[r.session];
        for (auto it = out.begin(); it != out.end() && it->first <= r.k;) {
            dhr_completion c{};
            c.request_id = it->second.id;
            c.session = r.session;
            c.frame = it->second.frame;
            c.t_arrival_ns = it->second.t_arrival;
            if (it->first == r.k) {
                c.t_start_ns = (uint64_t)((int64_t)r.t_start + L.clock_offset);
                c.t_done_ns = (uint64_t)((int64_t)r.t_done + L.clock_offset);
                c.batch_size = r.batch_size;
                ++s->n_frames;
            } else {
                c.t_done_ns = now_ns();
                c.dropped = 1;
                ++s->n_dropped;
            }
            s->done.push_back(c);
            it = out.erase(it);
        }
        if (r.t_start != last_batch) {
            ++s->n_batches;
            last_batch = r.t_start;
        }
    }
    __atomic_store_n(&L.ctl->ring_tail, tail, __ATOMIC_RELEASE);
}

// the loop's stream still has work (the graph launch has not ended) and the
// loop has not reported its end
static bool loop_running(const dhr_server* s) {
    if (!s->loop.active) return false;
    for (int li = 0; li < kLoops; ++li)
        if (__atomic_load_n(&s->loop.ctl->running[li], __ATOMIC_ACQUIRE) != 0u &&
            cudaStreamQuery(s->loop.stream[li]) == cudaErrorNotReady)
            return true;
    return false;
}

static std::array<uint64_t, kLoops> loop_epochs(const dhr_server* s) {
    std::array<uint64_t, kLoops> e;
    for (int li = 0; li < kLoops; ++li) e[li] = __atomic_load_n(&s->loop.ctl->epoch[li], __ATOMIC_ACQUIRE);
    return e;
}

// frees the memory of sessions closed while the loop ran, once no batch can
// still use it (two scheduling passes later, or the loop has ended)
static void release_session(dhr_server* s, int id);
static void loop_release_closed(dhr_server* s) {
    LoopHost& L = s->loop;
    const auto epoch = loop_epochs(s);
    const bool running = loop_running(s);
    auto& v = L.to_release;
    for (size_t i = 0; i < v.size();) {
        bool safe = true;
        for (int li = 0; li < kLoops; ++li)
            safe = safe && (__atomic_load_n(&L.ctl->running[li], __ATOMIC_ACQUIRE) == 0u ||
                            epoch[li] >= v[i].second[li] + 2);
        if (!running || safe) {
            release_session(s, v[i].first);
            v.erase(v.begin() + i);
        } else {
            ++i;
        }
    }
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

extern "C" dhr_status dhr_server_loop_stop(dhr_server* s);

extern "C" void dhr_server_destroy(dhr_server* s) {
    if (!s) return;
    if (s->loop.active) dhr_server_loop_stop(s);
    loop_destroy(s->loop);
    for (auto& sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.graph) cudaGraphExecDestroy(sl.graph);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFreeHost(sl.h_table);
        cudaFree(sl.d_table);
    }
    for (auto& se : s->sessions)
        if (se.mem) cudaFreeAsync(se.mem, s->mem_stream);
    if (s->mem_stream) {
        cudaStreamSynchronize(s->mem_stream);
        cudaStreamDestroy(s->mem_stream);
    }
    if (s->ref) cudaEventDestroy(s->ref);
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->fork_st) cudaStreamDestroy(s->fork_st);
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
    int least = 0, greatest = 0;
    if (cudaStreamCreateWithFlags(&s->mem_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s->fork_st, cudaStreamNonBlocking, least) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess)
        st = set_error(DHR_ERR_CUDA, "server_create: cannot create a stream");
    for (auto& sl : s->slots) {
        if (st != DHR_OK) break;
        int least = 0, greatest = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (!e) e = cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, greatest);
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
    if (st == DHR_OK) st = loop_create(s);
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
        if (s->sessions.size() >= (size_t)kLoopMaxSessions)
            return set_error(DHR_ERR_ADMISSION, "server_open: too many sessions (%d)", kLoopMaxSessions);
        s->sessions.emplace_back();
        id = (int)s->sessions.size() - 1;
    }
    Session& se = s->sessions[id];
    se = Session();
    char* base = nullptr;
    // stream-ordered allocation on the server's own stream: neither this nor
    // the release below synchronises the device, which would wait for a
    // running device loop
    DHR_CUDA_TRY(cudaMallocAsync((void**)&base, L.total, s->mem_stream));
    DHR_CUDA_TRY(cudaMemsetAsync(base, 0, L.total, s->mem_stream));
    DHR_CUDA_TRY(cudaStreamSynchronize(s->mem_stream));
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
    s->loop.outstanding[id].clear();
    publish_slot(s, id, true);
    *session_out = id;
    return DHR_OK;
}

static void release_session(dhr_server* s, int id) {
    Session& se = s->sessions[id];
    if (se.mem) cudaFreeAsync(se.mem, s->mem_stream);
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
    LoopHost& L = s->loop;
    publish_slot(s, id, false);
    for (auto& kv : L.outstanding[id]) {     // published to the loop, never completed
        dhr_completion c{};
        c.request_id = kv.second.id;
        c.session = id;
        c.frame = kv.second.frame;
        c.t_arrival_ns = kv.second.t_arrival;
        c.t_done_ns = now_ns();
        c.dropped = 1;
        s->done.push_back(c);
        ++s->n_dropped;
    }
    L.outstanding[id].clear();
    if (loop_running(s)) {
        // a batch scheduled before the close may still use the buffers
        L.to_release.push_back({id, loop_epochs(s)});
        return DHR_OK;
    }
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
    if (s->loop.active) {   // the loop takes the newest request of the mailbox
        Request r;
        r.id = request_id;
        r.session = id;
        r.cam = *cam;
        r.warp = cam_target != nullptr;
        r.cam_target = cam_target ? *cam_target : *cam;
        r.frame = frame;
        r.t_arrival = t_arrival_ns;
        publish_request(s, id, r);
        return DHR_OK;
    }
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

extern "C" dhr_status dhr_server_set_raster_min_pixels(dhr_server* s, uint64_t min_pixels) {
    clear_error();
    DHR_CHECK_ARG(s, "server_set_raster_min_pixels: null server");
    s->raster_min_px = min_pixels;
    return DHR_OK;
}

extern "C" dhr_status dhr_server_pump(dhr_server* s, int32_t* launched) {
    clear_error();
    DHR_CHECK_ARG(s, "server_pump: null server");
    if (launched) *launched = 0;
    if (s->loop.active) {      // the device loop schedules; collect its records
        loop_collect(s);
        loop_release_closed(s);
        return DHR_OK;
    }
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
        it.raster = s->tp.primary == DHR_PRIMARY_RASTER && px >= s->raster_min_px && s->scene->n_tris > 0 &&
                    make_raster(r.cam, it.g_cur, it.m_cur, 4, it.rc, it.bl);
        it.raster_tgt = it.warp && s->tp.primary == DHR_PRIMARY_RASTER && px >= s->raster_min_px &&
                        s->scene->n_tris > 0 && make_raster(r.cam_target, it.g_tgt, it.m_tgt, 4, it.rc_tgt, it.bl_tgt);
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
    if (s->loop.active) {
        loop_collect(s);
        loop_release_closed(s);
        // wait for a record, or for the loop to end
        while (wait && s->done.empty() && loop_running(s)) {
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            loop_collect(s);
        }
        if (wait && s->done.empty() && !loop_running(s)) {
            loop_collect(s);
            bool timed_out = false;
            for (int li = 0; li < kLoops; ++li)
                timed_out = timed_out ||
                            __atomic_load_n(&s->loop.ctl->status[li], __ATOMIC_ACQUIRE) == (uint32_t)DHR_ERR_TIMEOUT;
            if (s->done.empty() && timed_out)
                return set_error(DHR_ERR_TIMEOUT, "server_poll: the device loop ended after its idle limit "
                                                  "without a request");
        }
    } else {
        DHR_TRY(reap(s, wait != 0 && s->done.empty()));
    }
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

extern "C" dhr_status dhr_server_read_output(dhr_server* s, int32_t id, float* ao_host, float* shadow_host) {
    clear_error();
    DHR_CHECK_ARG(s && ao_host && shadow_host, "server_read_output: null pointer");
    DHR_CHECK_ARG(id >= 0 && id < (int)s->sessions.size() && s->sessions[id].open, "server_read_output: bad session");
    const Session& se = s->sessions[id];
    const size_t bytes = (size_t)se.w * se.h * sizeof(float);
    DHR_CUDA_TRY(cudaMemcpyAsync(ao_host, se.fin_ao, bytes, cudaMemcpyDeviceToHost, s->mem_stream));
    DHR_CUDA_TRY(cudaMemcpyAsync(shadow_host, se.fin_sh, bytes, cudaMemcpyDeviceToHost, s->mem_stream));
    DHR_CUDA_TRY(cudaStreamSynchronize(s->mem_stream));
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

extern "C" dhr_status dhr_server_loop_start(dhr_server* s, uint32_t idle_ms, uint32_t max_run_ms) {
    clear_error();
    DHR_CHECK_ARG(s, "server_loop_start: null server");
    DHR_CHECK_ARG(!s->loop.active, "server_loop_start: the loop is already running");
    DHR_CHECK_ARG(idle_ms >= 1 && idle_ms <= 600000, "server_loop_start: idle_ms not in 1..600000");
    DHR_CHECK_ARG(max_run_ms >= 1 && max_run_ms <= 3600000, "server_loop_start: max_run_ms not in 1..3600000");
    LoopHost& L = s->loop;
    // batches the host launched finish first; the loop continues every
    // session's history from where they left it
    for (auto& sl : s->slots)
        if (sl.in_flight) {
            DHR_CUDA_TRY(cudaEventSynchronize(sl.done));
            DHR_TRY(complete_slot(s, sl));
        }
    for (size_t i = 0; i < s->sessions.size(); ++i)
        if (s->sessions[i].closing) release_session(s, (int)i);
    std::vector<DevSession> ds(kLoopMaxSessions);
    for (size_t i = 0; i < s->sessions.size() && i < (size_t)kLoopMaxSessions; ++i) {
        const Session& se = s->sessions[i];
        DevSession& d = ds[i];
        d.generation = L.generation[i];
        d.taken = L.published[i];
        d.cur = se.cur;
        d.has_prev = se.has_prev ? 1 : 0;
        d.cam_prev = se.cam_prev;
    }
    DHR_CUDA_TRY(cudaMemcpy(L.d_sess, ds.data(), sizeof(DevSession) * kLoopMaxSessions, cudaMemcpyHostToDevice));
    LoopMeta m;
    memset(&m, 0, sizeof(m));
    dhr_camera c0{};
    c0.width = c0.height = 1;
    m.tk_base = make_trace_consts(c0, s->tp);
    m.sk_base = make_consts(1, 1, &s->sp);
    m.levels = (int)s->sp.levels;
    m.nsq = s->sp.sigma_n == 128.0f ? 7 : -1;
    m.raster_min_px = (s->tp.primary == DHR_PRIMARY_RASTER && s->scene->n_tris > 0) ? s->raster_min_px : ~0ull;
    m.lim.idle_ns = (uint64_t)idle_ms * 1000000ull;
    m.lim.max_run_ns = (uint64_t)max_run_ms * 1000000ull;
    m.lim.poll_ns = 50000;                  // 50 us of waiting per scheduling pass
    m.lim.max_iters = (uint64_t)max_run_ms * 200ull + 1000ull;
    for (int li = 0; li < kLoops; ++li)
        DHR_CUDA_TRY(cudaMemcpy(L.d_meta[li], &m, sizeof(m), cudaMemcpyHostToDevice));
    DHR_CUDA_TRY(cudaMemset(L.d_shared, 0, sizeof(LoopShared)));
    memset(L.ring, 0, sizeof(LoopRecord) * kRingRecords);
    L.ctl->stop = 0;
    L.ctl->ring_tail = 0;
    L.ctl->max_batch_px = s->max_batch_px;
    L.ctl->n_slots = (uint32_t)std::min<size_t>(s->sessions.size(), (size_t)kLoopMaxSessions);
    for (int li = 0; li < kLoops; ++li) {
        L.ctl->epoch[li] = 0;
        L.ctl->status[li] = (uint32_t)DHR_OK;
        __atomic_store_n(&L.ctl->running[li], 1u, __ATOMIC_RELEASE);
    }
    // the newest queued request of each session moves into its mailbox
    for (size_t i = 0; i < s->sessions.size(); ++i) {
        Session& se = s->sessions[i];
        if (se.open && se.pending) {
            se.pending = false;
            publish_request(s, (int)i, se.req);
        }
    }
    s->order.clear();
    // device clock against the host clock
    uint64_t* clock_d = nullptr;
    DHR_CUDA_TRY(cudaHostGetDevicePointer((void**)&clock_d, L.clock, 0));
    const uint64_t h0 = now_ns();
    clock_kernel<<<1, 1, 0, L.stream[0]>>>(clock_d);
    DHR_CUDA_TRY(cudaGetLastError());
    DHR_CUDA_TRY(cudaStreamSynchronize(L.stream[0]));
    const uint64_t h1 = now_ns();
    L.clock_offset = (int64_t)((h0 + h1) / 2) - (int64_t)*(volatile uint64_t*)L.clock;
    for (int li = 0; li < kLoops; ++li) DHR_CUDA_TRY(cudaGraphLaunch(L.exec[li], L.stream[li]));
    L.active = true;
    return DHR_OK;
}

extern "C" dhr_status dhr_server_loop_stop(dhr_server* s) {
    clear_error();
    DHR_CHECK_ARG(s, "server_loop_stop: null server");
    LoopHost& L = s->loop;
    if (!L.active) return DHR_OK;
    __atomic_store_n(&L.ctl->stop, 1u, __ATOMIC_RELEASE);
    cudaError_t e = cudaSuccess;
    for (int li = 0; li < kLoops; ++li) {
        const cudaError_t ei = cudaStreamSynchronize(L.stream[li]);
        if (e == cudaSuccess) e = ei;
    }
    L.active = false;
    if (e != cudaSuccess) return set_error(DHR_ERR_CUDA, "server_loop_stop: %s", cudaGetErrorString(e));
    // records, then the loop's per-session state back to the host
    s->loop.active = true;
    loop_collect(s);
    s->loop.active = false;
    std::vector<DevSession> ds(kLoopMaxSessions);
    DHR_CUDA_TRY(cudaMemcpy(ds.data(), L.d_sess, sizeof(DevSession) * kLoopMaxSessions, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < s->sessions.size() && i < (size_t)kLoopMaxSessions; ++i) {
        Session& se = s->sessions[i];
        if (!se.open || ds[i].generation != L.generation[i]) continue;
        se.cur = ds[i].cur;
        se.has_prev = ds[i].has_prev != 0;
        se.cam_prev = ds[i].cam_prev;
        // requests the loop did not take: the newest is queued for the host's
        // batches, older ones were replaced (dropped)
        auto& out = L.outstanding[i];
        while (!out.empty() && out.begin()->first <= ds[i].taken) out.erase(out.begin());
        while (out.size() > 1) {
            dhr_completion c{};
            c.request_id = out.begin()->second.id;
            c.session = (int)i;
            c.frame = out.begin()->second.frame;
            c.t_arrival_ns = out.begin()->second.t_arrival;
            c.t_done_ns = now_ns();
            c.dropped = 1;
            s->done.push_back(c);
            ++s->n_dropped;
            out.erase(out.begin());
        }
        if (!out.empty()) {
            se.pending = true;
            se.req = out.begin()->second;
            s->order.push_back((int)i);
            L.published[i] = ds[i].taken;       // the mailbox request is withdrawn
            __atomic_store_n(&L.mb[i].seq, 2u * ds[i].taken, __ATOMIC_RELEASE);
            out.clear();
        }
    }
    for (auto& v : L.to_release) release_session(s, v.first);
    L.to_release.clear();
    bool timed_out = false;
    for (int li = 0; li < kLoops; ++li)
        timed_out = timed_out || __atomic_load_n(&L.ctl->status[li], __ATOMIC_ACQUIRE) == (uint32_t)DHR_ERR_TIMEOUT;
    if (timed_out)
        return set_error(DHR_ERR_TIMEOUT, "server_loop_stop: the device loop had ended at its idle or run-time limit");
    return DHR_OK;
}

extern "C" dhr_status dhr_server_loop_status(dhr_server* s, int32_t* running, uint64_t* batches) {
    clear_error();
    DHR_CHECK_ARG(s && running, "server_loop_status: null pointer");
    // from the flags the loop writes (no CUDA call)
    int r = 0;
    uint64_t b = 0;
    for (int li = 0; li < kLoops; ++li) {
        r |= (s->loop.active && __atomic_load_n(&s->loop.ctl->running[li], __ATOMIC_ACQUIRE) != 0u) ? 1 : 0;
        b += __atomic_load_n(&s->loop.ctl->epoch[li], __ATOMIC_ACQUIRE);
    }
    *running = r;
    if (batches) *batches = b;
    return DHR_OK;
}
