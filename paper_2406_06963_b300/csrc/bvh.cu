// LBVH construction on the device.
//
// Section 3.2 relies on grouping the scene hierarchically into bounding
// volumes so that most rays skip most geometry.  B300 has no ray-tracing
// cores, so the hierarchy is built here: Morton codes of triangle centroids
// (63 bits, 21 per axis), a device radix sort, the parallel binary radix
// tree construction of Karras ("Maximizing Parallelism in the Construction
// of BVHs, Octrees, and k-d Trees", HPG 2012), and a bottom-up box refit in
// which the second thread to reach a node computes its box.
#include <algorithm>
#include <cmath>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "common.cuh"

namespace dhr {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t float_flip(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_unflip(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

struct Tri3 {
    float3 a, b, c;
};

__device__ __forceinline__ Tri3 load_tri(const float* v, const uint32_t* idx, uint32_t t) {
    const uint32_t i0 = idx[3 * t], i1 = idx[3 * t + 1], i2 = idx[3 * t + 2];
    Tri3 r;
    r.a = make_float3(v[3 * i0], v[3 * i0 + 1], v[3 * i0 + 2]);
    r.b = make_float3(v[3 * i1], v[3 * i1 + 1], v[3 * i1 + 2]);
    r.c = make_float3(v[3 * i2], v[3 * i2 + 1], v[3 * i2 + 2]);
    return r;
}

// Validates indices and accumulates the centroid bounds (order-preserving
// integer encoding so that atomicMin/Max work on floats).
__global__ void centroid_bounds_kernel(const float* v, const uint32_t* idx, uint32_t n_tris,
                                       uint32_t n_verts, uint32_t* bounds /*[6] flipped*/,
                                       uint32_t* bad_index) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tris; t += gridDim.x * blockDim.x) {
        const uint32_t i0 = idx[3 * t], i1 = idx[3 * t + 1], i2 = idx[3 * t + 2];
        if (i0 >= n_verts || i1 >= n_verts || i2 >= n_verts) {
            atomicExch(bad_index, 1u);
            continue;
        }
        const Tri3 r = load_tri(v, idx, t);
        const float c[3] = {(r.a.x + r.b.x + r.c.x) * (1.0f / 3.0f), (r.a.y + r.b.y + r.c.y) * (1.0f / 3.0f),
                            (r.a.z + r.b.z + r.c.z) * (1.0f / 3.0f)};
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], c[k]);
            hi[k] = fmaxf(hi[k], c[k]);
        }
    }
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&bounds[k], float_flip(lo[k]));
            atomicMax(&bounds[3 + k], float_flip(hi[k]));
        }
    }
}

__device__ __forceinline__ uint64_t spread21(uint32_t x) {
    uint64_t v = x & 0x1FFFFFu;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__global__ void morton_kernel(const float* v, const uint32_t* idx, uint32_t n_tris,
                              const uint32_t* bounds, uint64_t* keys, uint32_t* values) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tris) return;
    const Tri3 r = load_tri(v, idx, t);
    const float c[3] = {(r.a.x + r.b.x + r.c.x) * (1.0f / 3.0f), (r.a.y + r.b.y + r.c.y) * (1.0f / 3.0f),
                        (r.a.z + r.b.z + r.c.z) * (1.0f / 3.0f)};
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
        const float lo = float_unflip(bounds[k]), hi = float_unflip(bounds[3 + k]);
        const float ext = hi - lo;
        float u = ext > 0.0f ? (c[k] - lo) / ext : 0.5f;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        q[k] = min((uint32_t)(u * 2097152.0f), 2097151u);
    }
    keys[t] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
    values[t] = t;
}

// Longest common prefix of keys i and j (index bits break ties); -1 outside.
__device__ __forceinline__ int delta(const uint64_t* keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint64_t a = keys[i], b = keys[j];
    if (a == b) return 64 + __clz((uint32_t)i ^ (uint32_t)j);
    return __clzll(a ^ b);
}

// Karras 2012: internal node i covers a key range [first, last] found by an
// exponential then binary search; its split is the highest differing bit.
__global__ void karras_kernel(const uint64_t* keys, int n, int2* children, int* parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(keys, n, i, i - d);
    int lmax = 2;
    while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(keys, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int gamma = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const int c0 = (lo == gamma) ? ~gamma : gamma;          // leaf refs are ~index
    const int c1 = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    children[i] = make_int2(c0, c1);
    parent[c0 >= 0 ? c0 : (n - 1) + ~c0] = i;
    parent[c1 >= 0 ? c1 : (n - 1) + ~c1] = i;
}

// Node slots 0..n-2 internal, n-1.. leaves.
__device__ __forceinline__ int slot_of(int ref, int n) { return ref >= 0 ? ref : (n - 1) + ~ref; }

// Leaves: write sorted triangle data and leaf boxes, then climb.  The second
// thread to arrive at a node computes its box and height and goes on.
__global__ void refit_kernel(const float* v, const uint32_t* idx, const uint32_t* mesh,
                             const uint32_t* order, int n, const int2* children, const int* parent,
                             float4* lo, float4* hi, int* height, uint32_t* visits, float4* tris) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t t = order[k];
    const Tri3 r = load_tri(v, idx, t);
    tris[3 * k + 0] = make_float4(r.a.x, r.a.y, r.a.z, __uint_as_float(t));
    tris[3 * k + 1] = make_float4(r.b.x, r.b.y, r.b.z, __uint_as_float(mesh ? mesh[t] : 0u));
    tris[3 * k + 2] = make_float4(r.c.x, r.c.y, r.c.z, 0.0f);
    const int leaf = (n - 1) + k;
    lo[leaf] = make_float4(fminf(r.a.x, fminf(r.b.x, r.c.x)), fminf(r.a.y, fminf(r.b.y, r.c.y)),
                           fminf(r.a.z, fminf(r.b.z, r.c.z)), 0.0f);
    hi[leaf] = make_float4(fmaxf(r.a.x, fmaxf(r.b.x, r.c.x)), fmaxf(r.a.y, fmaxf(r.b.y, r.c.y)),
                           fmaxf(r.a.z, fmaxf(r.b.z, r.c.z)), 0.0f);
    height[leaf] = 0;
    if (n == 1) return;
    int node = parent[leaf];
    for (int level = 0; level < 4096; ++level) {   // a tree deeper than this is rejected below
        __threadfence();
        if (atomicAdd(&visits[node], 1u) == 0u) return;   // sibling not done yet
        __threadfence();
        const int2 ch = children[node];
        const int a = slot_of(ch.x, n), b = slot_of(ch.y, n);
        const float4 la = __ldcg(&lo[a]), lb = __ldcg(&lo[b]);
        const float4 ha = __ldcg(&hi[a]), hb = __ldcg(&hi[b]);
        lo[node] = make_float4(fminf(la.x, lb.x), fminf(la.y, lb.y), fminf(la.z, lb.z), 0.0f);
        hi[node] = make_float4(fmaxf(ha.x, hb.x), fmaxf(ha.y, hb.y), fmaxf(ha.z, hb.z), 0.0f);
        height[node] = 1 + max(__ldcg(&height[a]), __ldcg(&height[b]));
        if (node == 0) return;
        node = parent[node];
    }
    height[0] = 1 << 20;   // climb did not reach the root: flag a corrupt tree
}

__global__ void pack_kernel(int n, const int2* children, const float4* lo, const float4* hi,
                            float4* nodes) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int2 ch = children[i];
    const int a = slot_of(ch.x, n), b = slot_of(ch.y, n);
    const float4 la = lo[a], ha = hi[a], lb = lo[b], hb = hi[b];
    nodes[4 * i + 0] = make_float4(la.x, lb.x, ha.x, hb.x);
    nodes[4 * i + 1] = make_float4(la.y, lb.y, ha.y, hb.y);
    nodes[4 * i + 2] = make_float4(la.z, lb.z, ha.z, hb.z);
    nodes[4 * i + 3] = make_float4(__int_as_float(ch.x), __int_as_float(ch.y), 0.0f, 0.0f);
}

// One triangle: a root node whose two children are the same leaf.
__global__ void single_kernel(const float* v, const uint32_t* idx, const uint32_t* mesh,
                              float4* nodes, float4* tris) {
    const Tri3 r = load_tri(v, idx, 0);
    tris[0] = make_float4(r.a.x, r.a.y, r.a.z, __uint_as_float(0u));
    tris[1] = make_float4(r.b.x, r.b.y, r.b.z, __uint_as_float(mesh ? mesh[0] : 0u));
    tris[2] = make_float4(r.c.x, r.c.y, r.c.z, 0.0f);
    const float lx = fminf(r.a.x, fminf(r.b.x, r.c.x)), hx = fmaxf(r.a.x, fmaxf(r.b.x, r.c.x));
    const float ly = fminf(r.a.y, fminf(r.b.y, r.c.y)), hy = fmaxf(r.a.y, fmaxf(r.b.y, r.c.y));
    const float lz = fminf(r.a.z, fminf(r.b.z, r.c.z)), hz = fmaxf(r.a.z, fmaxf(r.b.z, r.c.z));
    nodes[0] = make_float4(lx, lx, hx, hx);
    nodes[1] = make_float4(ly, ly, hy, hy);
    nodes[2] = make_float4(lz, lz, hz, hz);
    nodes[3] = make_float4(__int_as_float(~0), __int_as_float(~0), 0.0f, 0.0f);
}

// ---------------------------------------------------------------- PLOC
// Parallel locally-ordered clustering (Meister & Bittner, "Parallel
// Locally-Ordered Clustering for Bounding Volume Hierarchy Construction",
// IEEE TVCG 2018): clusters stay in Morton order; each finds, within a
// window of +-r positions, the neighbour whose merged box has the smallest
// surface area; mutual nearest neighbours merge into a new node; the array
// is compacted; repeat until one cluster remains.

__device__ __forceinline__ float half_area(float4 lo, float4 hi) {
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

__device__ __forceinline__ float4 fmin4(float4 a, float4 b) {
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), 0.f);
}
__device__ __forceinline__ float4 fmax4(float4 a, float4 b) {
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), 0.f);
}

// sorted triangle data + one cluster per leaf
__global__ void ploc_leaves_kernel(const float* v, const uint32_t* idx, const uint32_t* mesh, const uint32_t* order,
                                   int n, float4* tris, int* cl_ref, float4* cl_lo, float4* cl_hi,
                                   float4* leaf_lo, float4* leaf_hi) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t t = order[k];
    const Tri3 r = load_tri(v, idx, t);
    tris[3 * k + 0] = make_float4(r.a.x, r.a.y, r.a.z, __uint_as_float(t));
    tris[3 * k + 1] = make_float4(r.b.x, r.b.y, r.b.z, __uint_as_float(mesh ? mesh[t] : 0u));
    tris[3 * k + 2] = make_float4(r.c.x, r.c.y, r.c.z, 0.0f);
    const float4 lo = make_float4(fminf(r.a.x, fminf(r.b.x, r.c.x)), fminf(r.a.y, fminf(r.b.y, r.c.y)),
                                  fminf(r.a.z, fminf(r.b.z, r.c.z)), 0.0f);
    const float4 hi = make_float4(fmaxf(r.a.x, fmaxf(r.b.x, r.c.x)), fmaxf(r.a.y, fmaxf(r.b.y, r.c.y)),
                                  fmaxf(r.a.z, fmaxf(r.b.z, r.c.z)), 0.0f);
    cl_ref[k] = ~k;
    cl_lo[k] = lo;
    cl_hi[k] = hi;
    leaf_lo[k] = lo;
    leaf_hi[k] = hi;
}

// nearest neighbour by merged surface area within +-r (ties: smaller index)
__global__ void ploc_nn_kernel(int C, int r, const float4* lo, const float4* hi, int* nn) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const float4 li = lo[i], hi_ = hi[i];
    float best = INFINITY;
    int bj = -1;
    const int j0 = max(0, i - r), j1 = min(C - 1, i + r);
    for (int j = j0; j <= j1; ++j) {
        if (j == i) continue;
        const float d = half_area(fmin4(li, __ldg(lo + j)), fmax4(hi_, __ldg(hi + j)));
        if (d < best || (d == best && j < bj)) {
            best = d;
            bj = j;
        }
    }
    nn[i] = bj;
}

// merge flag (the smaller index of a mutual pair creates the node) and
// survive flag (the larger index of a mutual pair disappears)
__global__ void ploc_flags_kernel(int C, const int* nn, int* merge, int* keep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C) return;
    const int j = nn[i];
    const bool mutual = j >= 0 && nn[j] == i;
    merge[i] = (mutual && i < j) ? 1 : 0;
    keep[i] = (mutual && i > j) ? 0 : 1;
}

__device__ __forceinline__ int ref_height(int ref, const int* nheight) { return ref < 0 ? 0 : nheight[ref]; }

// create the merged nodes and scatter the surviving clusters, in order
__global__ void ploc_merge_kernel(int C, const int* nn, const int* merge, const int* merge_ofs, const int* keep,
                                  const int* keep_ofs, int node_base, const int* cl_ref, const float4* cl_lo,
                                  const float4* cl_hi, int2* children, float4* nlo, float4* nhi, int* nheight,
                                  int* out_ref, float4* out_lo, float4* out_hi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C || !keep[i]) return;
    int ref = cl_ref[i];
    float4 lo = cl_lo[i], hi = cl_hi[i];
    if (merge[i]) {
        const int j = nn[i];
        const int node = node_base + merge_ofs[i];
        const int rj = cl_ref[j];
        lo = fmin4(lo, cl_lo[j]);
        hi = fmax4(hi, cl_hi[j]);
        children[node] = make_int2(ref, rj);
        nlo[node] = lo;
        nhi[node] = hi;
        nheight[node] = 1 + max(ref_height(ref, nheight), ref_height(rj, nheight));
        ref = node;
    }
    const int o = keep_ofs[i];
    out_ref[o] = ref;
    out_lo[o] = lo;
    out_hi[o] = hi;
}

// creation order m (root = n - 2, created last) -> traversal order n-2-m (root = 0)
__global__ void ploc_pack_kernel(int n, const int2* children, const float4* nlo, const float4* nhi,
                                 const float4* leaf_lo, const float4* leaf_hi, float4* nodes) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n - 1) return;
    const int2 ch = children[m];
    const int refs[2] = {ch.x, ch.y};
    float4 lo[2], hi[2];
    int out_ref[2];
    for (int c = 0; c < 2; ++c) {
        const int r = refs[c];
        if (r < 0) {
            lo[c] = leaf_lo[~r];
            hi[c] = leaf_hi[~r];
            out_ref[c] = r;
        } else {
            lo[c] = nlo[r];
            hi[c] = nhi[r];
            out_ref[c] = (n - 2) - r;
        }
    }
    const int i = (n - 2) - m;
    nodes[4 * i + 0] = make_float4(lo[0].x, lo[1].x, hi[0].x, hi[1].x);
    nodes[4 * i + 1] = make_float4(lo[0].y, lo[1].y, hi[0].y, hi[1].y);
    nodes[4 * i + 2] = make_float4(lo[0].z, lo[1].z, hi[0].z, hi[1].z);
    nodes[4 * i + 3] = make_float4(__int_as_float(out_ref[0]), __int_as_float(out_ref[1]), 0.0f, 0.0f);
}

template <class T>
dhr_status dmalloc(T** p, size_t count, const char* what) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
    if (e != cudaSuccess)
        return set_error(e == cudaErrorMemoryAllocation ? DHR_ERR_OOM : DHR_ERR_CUDA,
                         "cudaMalloc(%s, %zu bytes): %s", what, count * sizeof(T),
                         cudaGetErrorString(e));
    return DHR_OK;
}

struct Scratch {
    uint32_t* bounds = nullptr;
    uint64_t* keys = nullptr;
    uint64_t* keys_sorted = nullptr;
    uint32_t* vals = nullptr;
    uint32_t* vals_sorted = nullptr;
    int2* children = nullptr;
    int* parent = nullptr;
    float4* lo = nullptr;
    float4* hi = nullptr;
    int* height = nullptr;
    uint32_t* visits = nullptr;
    void* cub_tmp = nullptr;
    // PLOC
    int* cl_ref[2] = {nullptr, nullptr};
    float4* cl_lo[2] = {nullptr, nullptr};
    float4* cl_hi[2] = {nullptr, nullptr};
    int* nn = nullptr;
    int* merge = nullptr;
    int* merge_ofs = nullptr;
    int* keep = nullptr;
    int* keep_ofs = nullptr;
    void* scan_tmp = nullptr;
    ~Scratch() {
        cudaFree(bounds); cudaFree(keys); cudaFree(keys_sorted); cudaFree(vals);
        cudaFree(vals_sorted); cudaFree(children); cudaFree(parent); cudaFree(lo);
        cudaFree(hi); cudaFree(height); cudaFree(visits); cudaFree(cub_tmp);
        for (int i = 0; i < 2; ++i) { cudaFree(cl_ref[i]); cudaFree(cl_lo[i]); cudaFree(cl_hi[i]); }
        cudaFree(nn); cudaFree(merge); cudaFree(merge_ofs); cudaFree(keep); cudaFree(keep_ofs);
        cudaFree(scan_tmp);
    }
};

// PLOC over the Morton-sorted leaves (s.vals_sorted); nodes in s.children,
// boxes in s.lo / s.hi ([0, n-1) internal, [n-1, 2n-1) leaves).
dhr_status build_ploc(const float* v, const uint32_t* idx, const uint32_t* mesh, int n, cudaStream_t st,
                      dhr_scene* sc, Scratch& s) {
    constexpr int kRadius = 32;
    for (int b = 0; b < 2; ++b) {
        DHR_TRY(dmalloc(&s.cl_ref[b], n, "clusters"));
        DHR_TRY(dmalloc(&s.cl_lo[b], n, "clusters"));
        DHR_TRY(dmalloc(&s.cl_hi[b], n, "clusters"));
    }
    DHR_TRY(dmalloc(&s.nn, n, "nn"));
    DHR_TRY(dmalloc(&s.merge, n, "merge"));
    DHR_TRY(dmalloc(&s.merge_ofs, n, "merge"));
    DHR_TRY(dmalloc(&s.keep, n, "keep"));
    DHR_TRY(dmalloc(&s.keep_ofs, n, "keep"));
    size_t scan_bytes = 0;
    DHR_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, s.merge, s.merge_ofs, n, st));
    DHR_CUDA_TRY(cudaMalloc(&s.scan_tmp, scan_bytes));
    float4* leaf_lo = s.lo + (n - 1);
    float4* leaf_hi = s.hi + (n - 1);
    ploc_leaves_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(
        v, idx, mesh, s.vals_sorted, n, sc->tris, s.cl_ref[0], s.cl_lo[0], s.cl_hi[0], leaf_lo, leaf_hi);
    DHR_CUDA_TRY(cudaGetLastError());
    int C = n, cur = 0, node_base = 0;
    for (int it = 0; C > 1; ++it) {
        if (it >= 4096) return set_error(DHR_ERR_CUDA, "create_scene: PLOC did not converge");
        const int g = (C + kThreads - 1) / kThreads;
        ploc_nn_kernel<<<g, kThreads, 0, st>>>(C, kRadius, s.cl_lo[cur], s.cl_hi[cur], s.nn);
        ploc_flags_kernel<<<g, kThreads, 0, st>>>(C, s.nn, s.merge, s.keep);
        DHR_CUDA_TRY(cudaGetLastError());
        DHR_CUDA_TRY(cub::DeviceScan::ExclusiveSum(s.scan_tmp, scan_bytes, s.merge, s.merge_ofs, C, st));
        DHR_CUDA_TRY(cub::DeviceScan::ExclusiveSum(s.scan_tmp, scan_bytes, s.keep, s.keep_ofs, C, st));
        ploc_merge_kernel<<<g, kThreads, 0, st>>>(C, s.nn, s.merge, s.merge_ofs, s.keep, s.keep_ofs, node_base,
                                                  s.cl_ref[cur], s.cl_lo[cur], s.cl_hi[cur], s.children, s.lo,
                                                  s.hi, s.height, s.cl_ref[cur ^ 1], s.cl_lo[cur ^ 1],
                                                  s.cl_hi[cur ^ 1]);
        DHR_CUDA_TRY(cudaGetLastError());
        int tail[4];
        DHR_CUDA_TRY(cudaMemcpyAsync(&tail[0], s.merge + C - 1, 4, cudaMemcpyDeviceToHost, st));
        DHR_CUDA_TRY(cudaMemcpyAsync(&tail[1], s.merge_ofs + C - 1, 4, cudaMemcpyDeviceToHost, st));
        DHR_CUDA_TRY(cudaMemcpyAsync(&tail[2], s.keep + C - 1, 4, cudaMemcpyDeviceToHost, st));
        DHR_CUDA_TRY(cudaMemcpyAsync(&tail[3], s.keep_ofs + C - 1, 4, cudaMemcpyDeviceToHost, st));
        DHR_CUDA_TRY(cudaStreamSynchronize(st));
        const int merges = tail[0] + tail[1], left = tail[2] + tail[3];
        if (merges == 0) return set_error(DHR_ERR_CUDA, "create_scene: PLOC made no progress");
        node_base += merges;
        C = left;
        cur ^= 1;
    }
    if (node_base != n - 1) return set_error(DHR_ERR_CUDA, "create_scene: PLOC built %d nodes for %d leaves",
                                             node_base, n);
    ploc_pack_kernel<<<(n - 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(n, s.children, s.lo, s.hi, leaf_lo,
                                                                            leaf_hi, sc->nodes);
    DHR_CUDA_TRY(cudaGetLastError());
    int h = 0;
    DHR_CUDA_TRY(cudaMemcpyAsync(&h, s.height + (n - 2), sizeof(int), cudaMemcpyDeviceToHost, st));
    DHR_CUDA_TRY(cudaStreamSynchronize(st));
    sc->height = (uint32_t)h;
    return DHR_OK;
}

}  // namespace

dhr_status build_lbvh(const float* v, const uint32_t* idx, const uint32_t* mesh, uint32_t n_verts,
                      uint32_t n_tris, cudaStream_t st, dhr_scene* sc, uint32_t builder) {
    sc->n_tris = n_tris;
    if (n_tris == 0) return DHR_OK;
    cudaEvent_t e0, e1;
    DHR_CUDA_TRY(cudaEventCreate(&e0));
    DHR_CUDA_TRY(cudaEventCreate(&e1));
    DHR_CUDA_TRY(cudaEventRecord(e0, st));
    const int n = (int)n_tris;
    const int n_int = n > 1 ? n - 1 : 1;
    DHR_TRY(dmalloc(&sc->nodes, (size_t)4 * n_int, "bvh nodes"));
    DHR_TRY(dmalloc(&sc->tris, (size_t)3 * n, "bvh triangles"));
    sc->n_nodes = n_int;
    sc->bytes = (uint64_t)n_int * 64 + (uint64_t)n * 48;
    Scratch s;
    DHR_TRY(dmalloc(&s.bounds, 7, "bounds"));
    {
        uint32_t init[7];
        for (int k = 0; k < 3; ++k) { init[k] = 0xFFFFFFFFu; init[3 + k] = 0u; }
        init[6] = 0u;
        DHR_CUDA_TRY(cudaMemcpyAsync(s.bounds, init, sizeof(init), cudaMemcpyHostToDevice, st));
    }
    const int grid = (n + kThreads - 1) / kThreads;
    centroid_bounds_kernel<<<min(grid, 148 * 8), kThreads, 0, st>>>(v, idx, n_tris, n_verts, s.bounds,
                                                                   s.bounds + 6);
    DHR_CUDA_TRY(cudaGetLastError());
    uint32_t bad = 0;
    DHR_CUDA_TRY(cudaMemcpyAsync(&bad, s.bounds + 6, 4, cudaMemcpyDeviceToHost, st));
    DHR_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad) return set_error(DHR_ERR_INVALID, "create_scene: a triangle index is >= n_vertices");
    if (n == 1) {
        single_kernel<<<1, 1, 0, st>>>(v, idx, mesh, sc->nodes, sc->tris);
        DHR_CUDA_TRY(cudaGetLastError());
        sc->height = 1;
    } else {
        DHR_TRY(dmalloc(&s.keys, n, "keys"));
        DHR_TRY(dmalloc(&s.keys_sorted, n, "keys"));
        DHR_TRY(dmalloc(&s.vals, n, "vals"));
        DHR_TRY(dmalloc(&s.vals_sorted, n, "vals"));
        DHR_TRY(dmalloc(&s.children, n - 1, "children"));
        DHR_TRY(dmalloc(&s.parent, 2 * n - 1, "parent"));
        DHR_TRY(dmalloc(&s.lo, 2 * n - 1, "lo"));
        DHR_TRY(dmalloc(&s.hi, 2 * n - 1, "hi"));
        DHR_TRY(dmalloc(&s.height, 2 * n - 1, "height"));
        DHR_TRY(dmalloc(&s.visits, n - 1, "visits"));
        DHR_CUDA_TRY(cudaMemsetAsync(s.visits, 0, sizeof(uint32_t) * (n - 1), st));
        morton_kernel<<<grid, kThreads, 0, st>>>(v, idx, n_tris, s.bounds, s.keys, s.vals);
        DHR_CUDA_TRY(cudaGetLastError());
        size_t tmp_bytes = 0;
        DHR_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, s.keys, s.keys_sorted, s.vals,
                                                     s.vals_sorted, n, 0, 63, st));
        DHR_CUDA_TRY(cudaMalloc(&s.cub_tmp, tmp_bytes));
        DHR_CUDA_TRY(cub::DeviceRadixSort::SortPairs(s.cub_tmp, tmp_bytes, s.keys, s.keys_sorted,
                                                     s.vals, s.vals_sorted, n, 0, 63, st));
        if (builder == DHR_BUILD_LBVH) {
            karras_kernel<<<(n - 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(s.keys_sorted, n,
                                                                                  s.children, s.parent);
            DHR_CUDA_TRY(cudaGetLastError());
            refit_kernel<<<grid, kThreads, 0, st>>>(v, idx, mesh, s.vals_sorted, n, s.children, s.parent,
                                                    s.lo, s.hi, s.height, s.visits, sc->tris);
            DHR_CUDA_TRY(cudaGetLastError());
            pack_kernel<<<(n - 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(n, s.children, s.lo, s.hi,
                                                                               sc->nodes);
            DHR_CUDA_TRY(cudaGetLastError());
            int h = 0;
            DHR_CUDA_TRY(cudaMemcpyAsync(&h, s.height, sizeof(int), cudaMemcpyDeviceToHost, st));
            DHR_CUDA_TRY(cudaStreamSynchronize(st));
            sc->height = (uint32_t)h;
        } else {
            DHR_TRY(build_ploc(v, idx, mesh, n, st, sc, s));
        }
    }
    DHR_CUDA_TRY(cudaEventRecord(e1, st));
    DHR_CUDA_TRY(cudaEventSynchronize(e1));
    DHR_CUDA_TRY(cudaEventElapsedTime(&sc->build_ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (sc->height >= (uint32_t)kStackSize)
        return set_error(DHR_ERR_INVALID,
                         "create_scene: BVH height %u exceeds the traversal stack (%d)", sc->height,
                         kStackSize);
    return DHR_OK;
}

// ------------------------------------------------ start cells of bounded rays
namespace {

// Internal nodes under which lies every triangle whose box overlaps
// [lo, hi]: from the root, each of kSeedSlots slots follows one subtree; a
// child whose box misses [lo, hi] is dropped, a node whose two child boxes
// both overlap it takes a second slot while one is free, and a slot with no
// free slot to split into keeps its node.  A slot never steps onto a leaf
// (it keeps the leaf's parent), so a ray reaches every leaf through the slab
// test of the leaf's box, as from the root: a triangle whose box the ray
// misses is never tested (the watertight test alone can accept a ray that
// grazes a zero-area triangle).  Returns the occupied slots.
__device__ uint32_t seed_frontier(const SceneView& sc, float3 lo, float3 hi, int (&node)[kSeedSlots]) {
    constexpr uint32_t kAll = (1u << kSeedSlots) - 1u;
#pragma unroll
    for (int s = 0; s < kSeedSlots; ++s) node[s] = kSeedEmpty;
    if (sc.n_tris == 0) return 0u;
    node[0] = 0;
    uint32_t used = 1u, done = 0u;   // slots occupied / not to be split further
    // every round moves each open slot one level down: a tree of height
    // < kStackSize (checked at build) ends within kStackSize rounds
    for (int round = 0; round < kStackSize && (used & ~done); ++round) {
#pragma unroll
        for (int s = 0; s < kSeedSlots; ++s) {
            if (!(((used & ~done) >> s) & 1u)) continue;
            const int n = node[s];
            const float4* nd = sc.nodes + 4 * (int)dbg_index(n, sc.n_nodes, kSiteNode);
            const float4 a = nd[0], b = nd[1], c = nd[2], d = nd[3];
            const bool o0 = a.x <= hi.x && a.z >= lo.x && b.x <= hi.y && b.z >= lo.y && c.x <= hi.z && c.z >= lo.z;
            const bool o1 = a.y <= hi.x && a.w >= lo.x && b.y <= hi.y && b.w >= lo.y && c.y <= hi.z && c.w >= lo.z;
            const int c0 = __float_as_int(d.x), c1 = __float_as_int(d.y);
            if (o0 != o1) {
                const int c = o0 ? c0 : c1;
                if (c >= 0) node[s] = c;
                else done |= 1u << s;   // the one overlapping child is a leaf
            } else if (!o0) {
                node[s] = kSeedEmpty;
                used &= ~(1u << s);
                done = 0u;   // a slot came free: stopped slots may split again
            } else {
                const uint32_t fre = ~used & kAll;
                if (!fre || c0 < 0 || c1 < 0) {
                    done |= 1u << s;
                } else {
                    const int t = __ffs(fre) - 1;
                    node[s] = c0;
#pragma unroll
                    for (int u = 0; u < kSeedSlots; ++u)
                        if (u == t) node[u] = c1;
                    used |= 1u << t;
                }
            }
        }
    }
    return used;
}

// one thread per cell of every level
__global__ void seed_grid_kernel(SceneView sc, int4* cells) {
    const SeedGrid& g = sc.seeds;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.n_cells) return;
    int l = 0;
    while (l + 1 < g.levels && c >= g.off[l + 1]) ++l;
    const int r = c - g.off[l], dx = g.dim[l][0], dy = g.dim[l][1];
    const int i[3] = {r % dx, (r / dx) % dy, r / (dx * dy)};
    const float s = g.side[l];
    // the loose box, padded far beyond the rounding of its corners and of
    // the lookup's cell index
    const float pad = s * (1.0f / 1024.0f);
    float lo[3], hi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        lo[k] = g.org[k] + ((float)i[k] - 0.5f) * s - pad;
        hi[k] = g.org[k] + ((float)i[k] + 1.5f) * s + pad;
    }
    int node[kSeedSlots];
    seed_frontier(sc, make_float3(lo[0], lo[1], lo[2]), make_float3(hi[0], hi[1], hi[2]), node);
    static_assert(kSeedSlots == 4, "a cell is one int4");
    cells[c] = make_int4(node[0], node[1], node[2], node[3]);
}

}  // namespace

dhr_status build_seed_grid(dhr_scene* sc, cudaStream_t st) {
    SeedGrid& g = sc->seeds;
    g = SeedGrid{};
    if (sc->n_tris == 0) return DHR_OK;
    // the scene box: the root's two child boxes
    float4 root[4];
    DHR_CUDA_TRY(cudaMemcpyAsync(root, sc->nodes, sizeof(root), cudaMemcpyDeviceToHost, st));
    DHR_CUDA_TRY(cudaStreamSynchronize(st));
    const float lo[3] = {fminf(root[0].x, root[0].y), fminf(root[1].x, root[1].y), fminf(root[2].x, root[2].y)};
    const float hi[3] = {fmaxf(root[0].z, root[0].w), fmaxf(root[1].z, root[1].w), fmaxf(root[2].z, root[2].w)};
    float ext = 0.f;
    for (int k = 0; k < 3; ++k) ext = fmaxf(ext, hi[k] - lo[k]);
    if (!(ext > 0.f) || !std::isfinite(ext)) return DHR_OK;   // no grid: rays start at the root
    // level 0: 128 cells along the longest axis; each level's cells are
    // sqrt(2) times wider than the previous level's
    for (int k = 0; k < 3; ++k) {
        g.org[k] = lo[k];
        g.top[k] = hi[k];
    }
    long long total = 0;
    for (int l = 0; l < kSeedLevels; ++l) {
        const double s = (double)ext / 128.0 * std::pow(std::sqrt(2.0), (double)l);
        g.side[l] = (float)s;
        g.inv[l] = (float)(1.0 / s);
        bool one = true;
        for (int k = 0; k < 3; ++k) {
            g.dim[l][k] = std::max(1, (int)std::ceil((double)(hi[k] - lo[k]) / s));
            one = one && g.dim[l][k] == 1;
        }
        g.off[l] = (int)total;
        total += (long long)g.dim[l][0] * g.dim[l][1] * g.dim[l][2];
        g.levels = l + 1;
        if (one) break;
    }
    g.n_cells = (int)total;
    int4* cells = nullptr;
    DHR_TRY(dmalloc(&cells, (size_t)total, "seed grid"));
    g.cells = cells;
    sc->bytes += (uint64_t)total * sizeof(int4);
    seed_grid_kernel<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(sc->view(), cells);
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}

}  // namespace dhr
