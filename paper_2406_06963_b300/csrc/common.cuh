// Internal declarations shared by the libdhrs translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "dhrs.h"

namespace dhr {

// ---------------------------------------------------------------- errors
dhr_status set_error(dhr_status s, const char* fmt, ...);
void clear_error();

#define DHR_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::dhr::set_error(e_ == cudaErrorMemoryAllocation ? DHR_ERR_OOM       \
                                                                    : DHR_ERR_CUDA,     \
                                    "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),    \
                                    __FILE__, __LINE__);                                \
    } while (0)

#define DHR_CHECK_ARG(cond, ...)                                                        \
    do {                                                                                \
        if (!(cond)) return ::dhr::set_error(DHR_ERR_INVALID, __VA_ARGS__);             \
    } while (0)

#define DHR_TRY(expr)                     \
    do {                                  \
        dhr_status s_ = (expr);           \
        if (s_ != DHR_OK) return s_;      \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------ debug build
// Built with DHR_DEBUG (libdhrs_debug.so), every gather index at the checked
// sites is tested against its buffer's extent n.  An index outside [0, n)
// records the first such event of the translation unit in its error word
// (bit 63 set, the site in bits 40..47, the index's low 40 bits) and is
// replaced by 0, so the access stays inside the buffer (every checked buffer
// has n >= 1) and the kernel runs on.  dhr_debug_status collects and clears
// the words of all translation units.  Without DHR_DEBUG the check is the
// identity and costs nothing.
enum DebugSite : uint32_t {
    kSiteAtrousTap = 1,     // a-trous tap (colour and G-buffer)
    kSiteAtrousVar = 2,     // a-trous variance Gaussian
    kSiteDepthGrad = 3,     // depth slope neighbours
    kSiteReproject = 4,     // reprojection taps of the previous frame
    kSiteShortHist = 5,     // 7x7 short-history estimate
    kSiteNode = 6,          // BVH node fetch
    kSiteTriangle = 7,      // triangle fetch
    kSiteRasterList = 8,    // rasterised tile list words
    kSiteRasterBin = 9,     // binning writes
    kSiteAdjoint = 10,      // adjoint gathers and scatters
    kSiteSelfTest = 11,     // dhr_debug_selftest
    kSiteSeedCell = 12,     // start cell of a bounded ray
};

#ifdef DHR_DEBUG
static __device__ unsigned long long g_debug_err = 0;
#endif

__device__ __forceinline__ long long dbg_index(long long i, long long n, uint32_t site) {
#ifdef DHR_DEBUG
    if (i < 0 || i >= n) {
        atomicCAS(&g_debug_err, 0ull,
                  (1ull << 63) | ((unsigned long long)(site & 0xFFu) << 40) |
                      ((unsigned long long)i & 0xFFFFFFFFFFull));
        return 0;
    }
#else
    (void)n;
    (void)site;
#endif
    return i;
}

// host side: each translation unit registers a reader of its error word
using DebugReader = unsigned long long (*)();
void debug_register(DebugReader f);
#ifdef DHR_DEBUG
static unsigned long long debug_take_this_unit() {
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_debug_err, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(g_debug_err, &z, sizeof(z));
    }
    return v;
}
struct DebugRegistration {
    DebugRegistration() { debug_register(&debug_take_this_unit); }
};
static DebugRegistration g_debug_registration;
#endif

// ---------------------------------------------------------------- scene
// BVH node, 64 bytes: the boxes of both children plus their references,
// paired by plane so that one f32x2 fma gives both children's distances:
//   a = (c0.lo.x, c1.lo.x, c0.hi.x, c1.hi.x)
//   b = (c0.lo.y, c1.lo.y, c0.hi.y, c1.hi.y)
//   c = (c0.lo.z, c1.lo.z, c0.hi.z, c1.hi.z)
//   d = (child0, child1, -, -) as int bits; >= 0 internal node, < 0 leaf ~i
// Leaf i holds sorted triangle i: 3 float4 (v0, orig index bits),
// (v1, mesh id bits), (v2, 0).
//
// Start cells of bounded rays: a hierarchy of loose grids over the scene
// box.  Level l has cells of side s_l = s_0 sqrt(2)^l; cell i of an axis covers
// [org + (i - 1/2) s_l, org + (i + 3/2) s_l] (its own extent and half a side
// beyond each face), so a box of side <= s_l whose centre lies in cell i
// lies inside it.  A cell holds up to kSeedSlots nodes (kSeedEmpty: unused)
// under which lies every triangle whose box overlaps the cell's.
constexpr int kSeedSlots = 4, kSeedLevels = 16;
constexpr int kSeedEmpty = INT_MIN;
struct SeedGrid {
    const int4* cells;   // all levels' cells, level by level, x fastest, then y, then z
    float org[3];        // scene box minimum
    float top[3];        // scene box maximum
    float side[kSeedLevels];   // s_l
    float inv[kSeedLevels];    // 1 / s_l
    int levels;          // 0: no grid (every ray starts at the root)
    int n_cells;
    int dim[kSeedLevels][3];
    int off[kSeedLevels];
};

struct SceneView {
    const float4* nodes;
    const float4* tris;
    int32_t n_tris;
    const float4* chunk_box;   // per kChunk consecutive leaves: (lo, -), (hi, -) of their vertices
    int32_t n_nodes;           // internal nodes
    SeedGrid seeds;
};

// leaves per chunk of the rasteriser's frustum test (one binning block)
constexpr int kChunk = 128;

constexpr int kStackSize = 64;

// ------------------------------------------------ packed fp32x2 arithmetic
// Two binary32 values in one 64-bit register pair; the f32x2 instructions
// round each lane exactly as the scalar instruction would.
__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// Reduced-precision G-buffer element (DHR_FP16 form), 8 bytes: x = binary32
// linear depth, y = unit normal as two octahedral coordinates (Cigolle et
// al., "A Survey of Efficient Representations for Independent Unit
// Vectors", JCGT 2014) in 16-bit signed-normalised fixed point, q / 32767:
// the coordinates lie in [-1, 1], so fixed point spends all 16 bits on that
// range (binary16 would keep 11 bits of precision there and spend 5 on an
// exponent range that never occurs).  Depth stays binary32: the depth
// edge-stopping weight compares depth differences far below 16-bit
// resolution.
__device__ __forceinline__ float oct_sign(float v) { return v >= 0.0f ? 1.0f : -1.0f; }

__device__ __forceinline__ uint32_t snorm16(float v) {
    const int q = __float2int_rn(fminf(fmaxf(v, -1.0f), 1.0f) * 32767.0f);
    return (uint32_t)(q & 0xFFFF);
}

__device__ __forceinline__ float unsnorm16(uint32_t u) {
    return (float)(int16_t)(u & 0xFFFF) * (1.0f / 32767.0f);
}

__device__ __forceinline__ uint2 pack_gbuf16(float depth, float3 n) {
    const float s = fabsf(n.x) + fabsf(n.y) + fabsf(n.z);
    float ex = 0.0f, ey = 0.0f;
    if (s > 0.0f) {
        ex = n.x / s;
        ey = n.y / s;
        if (n.z < 0.0f) {
            const float tx = (1.0f - fabsf(ey)) * oct_sign(ex), ty = (1.0f - fabsf(ex)) * oct_sign(ey);
            ex = tx;
            ey = ty;
        }
    }
    return make_uint2(__float_as_uint(depth), snorm16(ex) | (snorm16(ey) << 16));
}

__device__ __forceinline__ float4 unpack_gbuf16(uint2 u) {
    const float ex = unsnorm16(u.y), ey = unsnorm16(u.y >> 16);
    float3 v = make_float3(ex, ey, 1.0f - fabsf(ex) - fabsf(ey));
    if (v.z < 0.0f) {
        const float tx = (1.0f - fabsf(ey)) * oct_sign(ex), ty = (1.0f - fabsf(ex)) * oct_sign(ey);
        v.x = tx;
        v.y = ty;
    }
    const float r = rsqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
    return make_float4(__uint_as_float(u.x), v.x * r, v.y * r, v.z * r);
}

}  // namespace dhr

struct dhr_scene {
    float4* nodes = nullptr;
    float4* tris = nullptr;
    float4* chunk_box = nullptr;
    dhr::SeedGrid seeds{};      // seeds.cells: device memory owned by the scene
    uint32_t n_tris = 0;
    uint32_t n_nodes = 0;
    uint32_t height = 0;
    uint64_t bytes = 0;
    float build_ms = 0.f;
    dhr::SceneView view() const {
        return dhr::SceneView{nodes, tris, (int32_t)n_tris, chunk_box, (int32_t)n_nodes, seeds};
    }
};

namespace dhr {

// ------------------------------------------------------------ entry points
dhr_status build_lbvh(const float* verts_d, const uint32_t* idx_d, const uint32_t* mesh_d,
                      uint32_t n_verts, uint32_t n_tris, cudaStream_t st, dhr_scene* sc, uint32_t builder);

// after_primary (optional): recorded on st once the primary pre-pass (if any)
// is enqueued, before the trace kernel
dhr_status launch_trace(const dhr_scene* sc, const dhr_camera* cam, const dhr_trace_params* p,
                        dhr_gbuffer* g, uint8_t* mask, uint8_t* ao, cudaStream_t st,
                        unsigned long long* stats = nullptr, cudaEvent_t after_primary = nullptr);

// dhr_trace_visibility's checks and launch, with launch_trace's event
dhr_status dhr_trace_visibility_events(const dhr_scene* scene, const dhr_camera* cam, const dhr_trace_params* params,
                                       dhr_gbuffer* gbuf_out, uint8_t* shadow_mask_out, uint8_t* ao_count_out,
                                       cudaStream_t st, cudaEvent_t after_primary);

dhr_status launch_trace_selective(const dhr_scene* sc, const dhr_camera* cam, const dhr_trace_params* p,
                                  const dhr_shadow_map* const* maps, dhr_gbuffer* g, uint8_t* mask, uint8_t* ao,
                                  uint8_t* ray_mask, cudaStream_t st);

// Rasterised primary visibility (raster.cu): leaves in the G-buffer's depth
// storage, per pixel, the key (t bits << 32 | original index) of the nearest
// hit of the pixel-centre ray, or ~0 where there is none.  Returns false (and
// launches nothing) when the camera basis is singular; the caller then traces
// primary rays instead.
dhr_status build_chunk_boxes(dhr_scene* sc, cudaStream_t st);
// the start cells of bounded rays (SeedGrid), after the BVH
dhr_status build_seed_grid(dhr_scene* sc, cudaStream_t st);
dhr_status launch_raster(const dhr_scene* sc, const dhr_camera* cam, dhr_gbuffer* g, cudaStream_t st,
                         bool* launched);

dhr_status check_trace_params(const dhr_trace_params* p);
dhr_status check_svgf_params(const dhr_svgf_params* p);

}  // namespace dhr
