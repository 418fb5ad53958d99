// Device code of the visibility trace, shared by the single-image kernels
// (trace.cu) and the batched serving kernels (serve.cu).
//
// cone-jittered shadow rays (Section 3.1) and radius-bounded cosine-weighted
// AO rays (Section 3.2, Eqs. 1-3), all by software traversal of the LBVH.
//
// Traversal: depth-first over the 2-wide BVH with a per-thread stack, near
// child first; any-hit rays stop at the first accepted hit, and AO rays
// carry tmax = r so that short rays prune most of the tree (Section 3.2).
// AO and shadow rays start below the root: at the nodes of a precomputed
// start cell that holds every triangle their segment can reach.
// Triangle test: the watertight ray/triangle intersection of Woop, Benthin
// and Wald (JCGT 2013) in binary32, with its double-precision fallback for
// edge functions that are exactly zero.  Ray/box test: slabs with the
// exit distance scaled by 1 + 2 gamma(3) (Ize, JCGT 2013) so that rounding
// never culls a box the ray touches.
#pragma once

#include <cuda_fp16.h>

#include <climits>
#include <cmath>

#include "common.cuh"
#include "sampling.cuh"

namespace dhr {

__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float comp(float3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

// Per-ray constants of the watertight test and of the slab test.
struct Ray {
    float3 o, d;
    unsigned long long idir2[3];   // per axis (1/d, 1/d), packed for f32x2 (tiny d clamped away from zero)
    unsigned long long noid2[3];   // per axis (-o/d, -o/d)
    int kx, ky, kz;
    float sx, sy, sz;
};

__device__ __forceinline__ Ray make_ray(float3 o, float3 d) {
    Ray r;
    r.o = o;
    r.d = d;
    const float eps = 1e-20f;
    const float dx = fabsf(d.x) > eps ? d.x : copysignf(eps, d.x);
    const float dy = fabsf(d.y) > eps ? d.y : copysignf(eps, d.y);
    const float dz = fabsf(d.z) > eps ? d.z : copysignf(eps, d.z);
    const float3 idir = make_float3(1.0f / dx, 1.0f / dy, 1.0f / dz);
    const float3 oidir = make_float3(o.x * idir.x, o.y * idir.y, o.z * idir.z);
    r.idir2[0] = pack2(idir.x, idir.x);
    r.idir2[1] = pack2(idir.y, idir.y);
    r.idir2[2] = pack2(idir.z, idir.z);
    r.noid2[0] = pack2(-oidir.x, -oidir.x);
    r.noid2[1] = pack2(-oidir.y, -oidir.y);
    r.noid2[2] = pack2(-oidir.z, -oidir.z);
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    r.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    r.kx = r.kz == 2 ? 0 : r.kz + 1;
    r.ky = r.kx == 2 ? 0 : r.kx + 1;
    if (comp(d, r.kz) < 0.0f) {
        const int t = r.kx;
        r.kx = r.ky;
        r.ky = t;
    }
    const float dkz = comp(d, r.kz);
    r.sx = comp(d, r.kx) / dkz;
    r.sy = comp(d, r.ky) / dkz;
    r.sz = 1.0f / dkz;
    return r;
}

// Watertight test; on a hit with tmin < t < tmax returns t and the scaled
// barycentrics (b0, b1, b2 of v0, v1, v2, summing to 1).
__device__ __forceinline__ bool hit_triangle(const Ray& r, float3 v0, float3 v1, float3 v2, float tmin,
                                             float tmax, float& t_out, float3& bary) {
    const float3 A = sub(v0, r.o), B = sub(v1, r.o), C = sub(v2, r.o);
    const float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
    const float Ax = comp(A, r.kx) - r.sx * Akz, Ay = comp(A, r.ky) - r.sy * Akz;
    const float Bx = comp(B, r.kx) - r.sx * Bkz, By = comp(B, r.ky) - r.sy * Bkz;
    const float Cx = comp(C, r.kx) - r.sx * Ckz, Cy = comp(C, r.ky) - r.sy * Ckz;
    float U = Cx * By - Cy * Bx;
    float V = Ax * Cy - Ay * Cx;
    float W = Bx * Ay - By * Ax;
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    const float det = U + V + W;
    if (det == 0.0f) return false;
    const float T = U * (r.sz * Akz) + V * (r.sz * Bkz) + W * (r.sz * Ckz);
    const float t = T / det;
    if (!(t > tmin && t < tmax)) return false;
    t_out = t;
    const float inv = 1.0f / det;
    bary = make_float3(U * inv, V * inv, W * inv);
    return true;
}

// three-operand min / max (one instruction on sm_100 and later)
__device__ __forceinline__ float max3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Slab tests of a node's two child boxes (node layout in common.cuh): the
// distances to both children's planes of an axis come from one f32x2 fma
// (each lane rounded once, as a scalar fma), then per child
// tn = max(near planes, tmin), tf = min(far planes, tmax); the exit distance
// is scaled by 1 + 2 gamma(3) (unit roundoff 2^-24) so that rounding never
// culls a box the ray touches.
__device__ __forceinline__ void slab2(const Ray& r, ulonglong2 ax, ulonglong2 ay, ulonglong2 az, float tmin,
                                      float tmax, float& e0, bool& h0, float& e1, bool& h1) {
    const float2 lx = unpack2(fma2(ax.x, r.idir2[0], r.noid2[0])), hx = unpack2(fma2(ax.y, r.idir2[0], r.noid2[0]));
    const float2 ly = unpack2(fma2(ay.x, r.idir2[1], r.noid2[1])), hy = unpack2(fma2(ay.y, r.idir2[1], r.noid2[1]));
    const float2 lz = unpack2(fma2(az.x, r.idir2[2], r.noid2[2])), hz = unpack2(fma2(az.y, r.idir2[2], r.noid2[2]));
    const float tn0 = max3(fminf(lx.x, hx.x), fminf(ly.x, hy.x), fmaxf(fminf(lz.x, hz.x), tmin));
    const float tf0 = min3(fmaxf(lx.x, hx.x), fmaxf(ly.x, hy.x), fminf(fmaxf(lz.x, hz.x), tmax));
    const float tn1 = max3(fminf(lx.y, hx.y), fminf(ly.y, hy.y), fmaxf(fminf(lz.y, hz.y), tmin));
    const float tf1 = min3(fmaxf(lx.y, hx.y), fmaxf(ly.y, hy.y), fminf(fmaxf(lz.y, hz.y), tmax));
    e0 = tn0;
    e1 = tn1;
    h0 = tn0 <= tf0 * 1.00000024f;
    h1 = tn1 <= tf1 * 1.00000024f;
}

// Closest hit (any_hit = false) or first hit (true) with tmin < t < tmax.
// Returns the sorted leaf index (or -1), t and barycentrics.  Ties in t
// go to the smaller original triangle index.
constexpr uint32_t kMaxSteps = 1u << 24;

// Work counters of one traversal (compiled in only by the statistics kernel).
struct Work {
    uint32_t visits = 0;   // internal nodes fetched (two child boxes tested each)
    uint32_t tests = 0;    // triangles tested
};

// The traversal starts at the root, or (kF > 0) at the nodes seed[s] of the
// slots s set in `seeds`, under which lies every triangle the ray can reach
// (seed_start).
template <bool kAnyHit, bool kStats = false, int kF = 0>
__device__ int traverse(const SceneView& sc, const Ray& r, float tmin, float& tmax, float3& bary,
                        int skip_leaf = -1, Work* work = nullptr, const int* seed = nullptr,
                        uint32_t seeds = 0) {
    if (sc.n_tris == 0) return -1;
    // a start from kF seeds holds up to kF - 1 of them on the stack beside
    // the at most height - 1 entries of a depth-first walk below depth 1
    int stack[kStackSize + kF];
    int sp = 0;
    int node = 0;
    if constexpr (kF > 0) {
        if (seeds == 0) return -1;
        bool first = true;
#pragma unroll
        for (int s = 0; s < kF; ++s) {
            if (!((seeds >> s) & 1u)) continue;
            if (first) node = seed[s];
            else stack[sp++] = seed[s];
            first = false;
        }
    }
    int best = -1;
    uint32_t best_orig = 0xFFFFFFFFu;
    // a valid tree visits each node at most once per ray; the cap only
    // guards against a corrupt tree
    for (uint32_t guard = 0; guard < kMaxSteps; ++guard) {
        if (node >= 0) {
            if (kStats) ++work->visits;
            node = (int)dbg_index(node, sc.n_nodes, kSiteNode);
            const ulonglong2* nd = reinterpret_cast<const ulonglong2*>(sc.nodes + 4 * node);
            const ulonglong2 ax = __ldg(nd), ay = __ldg(nd + 1), az = __ldg(nd + 2);
            const float4 d = __ldg(sc.nodes + 4 * node + 3);
            float e0, e1;
            bool h0, h1;
            slab2(r, ax, ay, az, tmin, tmax, e0, h0, e1, h1);
            int c0 = __float_as_int(d.x), c1 = __float_as_int(d.y);
            if (h0 && h1) {
                if (e1 < e0) {
                    const int t = c0;
                    c0 = c1;
                    c1 = t;
                }
                if (sp < kStackSize + kF) stack[sp++] = c1;   // height < kStackSize is checked at build
                node = c0;
                continue;
            }
            if (h0) { node = c0; continue; }
            if (h1) { node = c1; continue; }
        } else {
            const int leaf = (int)dbg_index(~node, sc.n_tris, kSiteTriangle);
            if (leaf == skip_leaf) goto pop;
            if (kStats) ++work->tests;
            const float4* tr = sc.tris + 3 * leaf;
            const float4 p0 = __ldg(tr), p1 = __ldg(tr + 1), p2 = __ldg(tr + 2);
            float t;
            float3 b;
            // closest hit admits t == tmax so that ties can go to the smaller index
            const float tlim = (kAnyHit || !(tmax < INFINITY)) ? tmax : __int_as_float(__float_as_int(tmax) + 1);
            if (hit_triangle(r, f3(p0), f3(p1), f3(p2), tmin, tlim, t, b)) {
                const uint32_t orig = __float_as_uint(p0.w);
                if (kAnyHit) {
                    tmax = t;
                    bary = b;
                    return leaf;
                }
                if (t < tmax || orig < best_orig) {
                    tmax = t;
                    bary = b;
                    best = leaf;
                    best_orig = orig;
                }
            }
        }
    pop:
        if (sp == 0) break;
        node = stack[--sp];
    }
    return best;
}

// Start of a bounded ray: the nodes of the start cell (SeedGrid) whose
// loose box contains the box [c - h, c + h] that the ray cannot leave.  The
// level is the finest whose cells are at least 2h wide (with a margin for
// the rounding of the cell index); a centre outside the grid takes the
// nearest cell, which still holds the part of the box inside the scene.
// Returns the occupied slots of seed; a box wider than every level (or not
// finite) starts at the root.
__device__ __forceinline__ uint32_t seed_start(const SceneView& sc, float3 c, float h, int (&seed)[kSeedSlots]) {
    const SeedGrid& g = sc.seeds;
    seed[0] = 0;
    const float w = 2.0f * h * 1.002f;
    int l = 0;
    while (l < g.levels && !(w <= g.side[l])) ++l;
    if (l == g.levels) return 1u;
    const float inv = g.inv[l];
    const int ix = min(max(__float2int_rd((c.x - g.org[0]) * inv), 0), g.dim[l][0] - 1);
    const int iy = min(max(__float2int_rd((c.y - g.org[1]) * inv), 0), g.dim[l][1] - 1);
    const int iz = min(max(__float2int_rd((c.z - g.org[2]) * inv), 0), g.dim[l][2] - 1);
    const long long cell = g.off[l] + ((long long)iz * g.dim[l][1] + iy) * g.dim[l][0] + ix;
    const int4 v = __ldg(g.cells + dbg_index(cell, g.n_cells, kSiteSeedCell));
    seed[0] = v.x;
    seed[1] = v.y;
    seed[2] = v.z;
    seed[3] = v.w;
    return (v.x != kSeedEmpty ? 1u : 0u) | (v.y != kSeedEmpty ? 2u : 0u) | (v.z != kSeedEmpty ? 4u : 0u) |
           (v.w != kSeedEmpty ? 8u : 0u);
}

// Start of an unbounded ray (a shadow ray): every triangle lies in the
// scene box, so the ray can reach only the part of it inside that box, up to
// its exit distance; the start cell is the one of that segment's box.
__device__ __forceinline__ uint32_t segment_start(const SceneView& sc, const Ray& r, int (&seed)[kSeedSlots]) {
    const SeedGrid& g = sc.seeds;
    seed[0] = 0;
    if (g.levels == 0) return 1u;
    const float o[3] = {r.o.x, r.o.y, r.o.z}, d[3] = {r.d.x, r.d.y, r.d.z};
    float t1 = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float id = unpack2(r.idir2[k]).x;   // 1 / d (tiny d clamped)
        t1 = fminf(t1, ((d[k] >= 0.0f ? g.top[k] : g.org[k]) - o[k]) * id);
    }
    t1 = fmaxf(t1, 0.0f);   // an origin outside the box, heading away: nothing to reach
    float c[3], h = 0.0f, m = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float e = fmaf(t1, d[k], o[k]);
        c[k] = 0.5f * (o[k] + e);
        h = fmaxf(h, fabsf(e - o[k]));
        m = fmaxf(m, fabsf(o[k]));
    }
    // half the widest side, padded far beyond the rounding of t1 and of e
    h = 0.5f * h + 1e-5f * (m + h);
    return seed_start(sc, make_float3(c[0], c[1], c[2]), h, seed);
}

// Unit normal of a triangle with a written binary32 operation order, each
// step rounded once (no fused multiply-add), the specification shared with
// the CPU oracle: a = v1 - v0, b = v2 - v0, c = a x b as (a_y b_z - a_z b_y,
// a_z b_x - a_x b_z, a_x b_y - a_y b_x), l = sqrt((c_x^2 + c_y^2) + c_z^2),
// n = c / l, square root and quotients correctly rounded.  The AO sample
// frame is built from the normal's sign bits (Duff et al.), which switch
// where a component is zero, so the bits must not depend on the compiler.
__device__ __forceinline__ float3 unit_normal_rn(float3 v0, float3 v1, float3 v2) {
    const float ax = __fsub_rn(v1.x, v0.x), ay = __fsub_rn(v1.y, v0.y), az = __fsub_rn(v1.z, v0.z);
    const float bx = __fsub_rn(v2.x, v0.x), by = __fsub_rn(v2.y, v0.y), bz = __fsub_rn(v2.z, v0.z);
    const float cx = __fsub_rn(__fmul_rn(ay, bz), __fmul_rn(az, by));
    const float cy = __fsub_rn(__fmul_rn(az, bx), __fmul_rn(ax, bz));
    const float cz = __fsub_rn(__fmul_rn(ax, by), __fmul_rn(ay, bx));
    const float q = __fadd_rn(__fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy)), __fmul_rn(cz, cz));
    const float l = __fsqrt_rn(q);
    return make_float3(__fdiv_rn(cx, l), __fdiv_rn(cy, l), __fdiv_rn(cz, l));
}

// Secondary-ray origin: the hit point moved along the normal by 16 units in
// the last place (binary32) of the largest vertex coordinate of the hit
// triangle -- an exact power of two, larger than the rounding error of the
// barycentric hit point -- so that the ray starts on the correct side of the
// surface.  The hit triangle itself is also skipped by secondary rays.
__device__ __forceinline__ float3 surface_origin(float3 X, float3 n, float3 v0, float3 v1, float3 v2) {
    float m = fmaxf(fmaxf(fmaxf(fabsf(v0.x), fabsf(v0.y)), fmaxf(fabsf(v0.z), fabsf(v1.x))),
                    fmaxf(fmaxf(fabsf(v1.y), fabsf(v1.z)), fmaxf(fmaxf(fabsf(v2.x), fabsf(v2.y)), fabsf(v2.z))));
    m = fmaxf(m, 9.5367431640625e-07f);                       // 2^-20
    const int e = (__float_as_int(m) >> 23) & 0xFF;            // biased exponent of m
    const float delta = __int_as_float((e - 19) << 23);        // 2^(e - 127 - 23 + 4)
    return make_float3(fmaf(delta, n.x, X.x), fmaf(delta, n.y, X.y), fmaf(delta, n.z, X.z));
}

struct TraceConsts {
    dhr_camera cam;
    float3 light[DHR_MAX_LIGHTS];
    float tan_cone[DHR_MAX_LIGHTS];
    uint32_t n_lights;
    float ao_radius;
    uint32_t ao_spp;
    uint32_t frame;
    uint32_t seed;
};

// trace constants of one frame; each light direction is normalised and the
// tan of each cone half angle computed in double on the host, each rounded
// once to binary32
inline TraceConsts make_trace_consts(const dhr_camera& cam, const dhr_trace_params& p) {
    TraceConsts k;
    k.cam = cam;
    for (uint32_t l = 0; l < DHR_MAX_LIGHTS; ++l) {
        if (l < p.n_lights) {
            const double lx = p.light_dir[l][0], ly = p.light_dir[l][1], lz = p.light_dir[l][2];
            const double n = std::sqrt(lx * lx + ly * ly + lz * lz);
            k.light[l] = make_float3((float)(lx / n), (float)(ly / n), (float)(lz / n));
            k.tan_cone[l] = (float)std::tan((double)p.cone_half_angle[l]);
        } else {
            k.light[l] = make_float3(0.f, 1.f, 0.f);
            k.tan_cone[l] = 0.f;
        }
    }
    k.n_lights = p.n_lights;
    k.ao_radius = p.ao_radius;
    k.ao_spp = p.ao_spp;
    k.frame = p.frame;
    k.seed = p.seed;
    return k;
}

// ------------------------------------------------ selective shadow rays
// Shadow map of one directional light (Section 5: a shadow map decides the
// pixels it can, a ray mask holds the rest).  Frame: unit L toward the
// light, eu, ev spanning the map plane; texel (i, j) has its centre at
// u0 + (i + 1/2) w along eu and v0 + (j + 1/2) w along ev; depth of a point
// x is h - L.x.  Level 0 is the R x R depth map (+inf where the texel ray
// meets nothing); level l (R >> l texels per side) holds the minimum over
// 2^l x 2^l texels, stored after level l - 1.
struct SmapView {
    const float* S;        // nullptr: this light is traced everywhere
    int res;
    float3 L, eu, ev;
    float u0, v0, w, inv_w, h;
    float zmin;            // minimum of level 0 (the top level)
    float tau;             // tan of the cone half angle
    float graze;           // sin of the cone half angle + kSmapGraze
};

struct SmapSet {
    SmapView m[DHR_MAX_LIGHTS];
};

constexpr int kClsTrace = 0, kClsLit = 1, kClsUmbra = 2;
constexpr float kSmapWindow = 4.0f;   // largest window radius r + 1 (texels)
constexpr double kSmapGraze = 0.05;   // margin of n.L over sin(cone half angle)

// offset of level l in a map of R x R texels: sum of (R >> k)^2, k < l
__host__ __device__ __forceinline__ size_t smap_level_offset(int R, int l) {
    const size_t s = (size_t)(R >> l);
    return 4 * ((size_t)R * R - s * s) / 3;
}

__device__ __forceinline__ int smap_clampi(float x, int hi) {
    return (int)fminf(fmaxf(x, 0.0f), (float)hi);
}

// Class of the receiver X (unit normal n facing the camera) for one light:
//  1. the cone lies below the surface (n.L < -g) -> umbra; it grazes the
//     surface (|n.L| <= g) -> trace;
//  2. a cone ray that has moved r texels sideways is at least r w / tan
//     closer to the light, so occluders met by the cone lie within
//     r0 = (z - zmin) tan / w texels; the minimum depth zocc over the 2 x 2
//     pyramid cells covering that range bounds the nearest occluder;
//  3. penumbra radius r = (z - zocc) tan / w texels; r + 1 > 4 -> trace;
//  4. each texel within r + 1 (Chebyshev) is occluded when its depth lies
//     more than one texel size above the receiver's tangent plane there;
//     all free -> lit, all occluded -> umbra, mixed -> trace.
__device__ __forceinline__ int smap_classify(const SmapView& m, float3 X, float3 n) {
    const float nL = dot(n, m.L);
    if (nL < -m.graze) return kClsUmbra;
    if (nL <= m.graze) return kClsTrace;
    const float a = (dot(m.eu, X) - m.u0) * m.inv_w - 0.5f;
    const float b = (dot(m.ev, X) - m.v0) * m.inv_w - 0.5f;
    const float z = m.h - dot(m.L, X);
    const int R1 = m.res - 1;
    const float r0 = fmaxf(0.0f, (z - m.zmin) * m.tau * m.inv_w);
    const int ilo = smap_clampi(floorf(a - r0), R1), ihi = smap_clampi(ceilf(a + r0), R1);
    const int jlo = smap_clampi(floorf(b - r0), R1), jhi = smap_clampi(ceilf(b + r0), R1);
    const int span = max(ihi - ilo, jhi - jlo) + 1;
    const int lv = 32 - __clz(span - 1);              // smallest l with 2^l >= span
    const float* M = m.S + smap_level_offset(m.res, lv);
    const int Rl = m.res >> lv;
    const int ci0 = ilo >> lv, ci1 = ihi >> lv, cj0 = jlo >> lv, cj1 = jhi >> lv;
    const float zocc = fminf(fminf(__ldg(M + (size_t)cj0 * Rl + ci0), __ldg(M + (size_t)cj0 * Rl + ci1)),
                             fminf(__ldg(M + (size_t)cj1 * Rl + ci0), __ldg(M + (size_t)cj1 * Rl + ci1)));
    const float r = fmaxf(0.0f, (z - zocc) * m.tau * m.inv_w);
    if (!(r + 1.0f <= kSmapWindow)) return kClsTrace;
    // at most 9 x 9 texels (r + 1 <= 4); the explicit cap also holds for
    // non-finite coordinates
    const int wi0 = smap_clampi(ceilf(a - r - 1.0f), R1), wi1 = min(smap_clampi(floorf(a + r + 1.0f), R1), wi0 + 8);
    const int wj0 = smap_clampi(ceilf(b - r - 1.0f), R1), wj1 = min(smap_clampi(floorf(b + r + 1.0f), R1), wj0 + 8);
    const float inv_nL = 1.0f / nL;
    const float gu = dot(n, m.eu) * inv_nL * m.w, gv = dot(n, m.ev) * inv_nL * m.w;
    bool occ = false, fre = false;
    for (int j = wj0; j <= wj1; ++j) {
        const float base = z + ((float)j - b) * gv - m.w;
        const float* row = m.S + (size_t)j * m.res;
        for (int i = wi0; i <= wi1; ++i) {
            const float plane = base + ((float)i - a) * gu;
            if (__ldg(row + i) < plane) occ = true;
            else fre = true;
        }
        if (occ && fre) return kClsTrace;
    }
    return occ ? kClsUmbra : kClsLit;
}

// Unnormalised direction of the ray through the centre of pixel (x, y), row 0
// at the top: D = forward + sx right + sy up, so that the ray parameter of a
// hit is its linear view depth.  Shared by the traced and the rasterised
// primary visibility so that both test the same ray.
__device__ __forceinline__ float3 primary_dir(const dhr_camera& c, int x, int y) {
    const int W = c.width, H = c.height;
    const float sx = (2.0f * (x + 0.5f) / W - 1.0f) * c.tan_half_fov_y * ((float)W / (float)H);
    const float sy = (1.0f - 2.0f * (y + 0.5f) / H) * c.tan_half_fov_y;
    return make_float3(c.forward[0] + sx * c.right[0] + sy * c.up[0],
                       c.forward[1] + sx * c.right[1] + sy * c.up[1],
                       c.forward[2] + sx * c.right[2] + sy * c.up[2]);
}

// ------------------------------------------ rasterised primary visibility
// The traversal only tests a triangle whose leaf box the ray passes (slab2).
// For a triangle of (near) zero area the watertight test's edge functions are
// rounding noise and could report a hit that the box test rules out, so such
// triangles take the same box test when rasterised (scalar form of slab2's
// lanes, with tmax = +inf: the traversal's tmax is the best hit so far, and a
// box beyond it holds no hit that could win).
__device__ __forceinline__ bool sliver(float3 v0, float3 v1, float3 v2) {
    const float3 e1 = sub(v1, v0), e2 = sub(v2, v0), c = cross(e1, e2);
    return !(dot(c, c) > 1e-12f * dot(e1, e1) * dot(e2, e2));
}

__device__ __forceinline__ bool leaf_box_hit(const Ray& r, float3 v0, float3 v1, float3 v2) {
    const float3 lo = make_float3(fminf(fminf(v0.x, v1.x), v2.x), fminf(fminf(v0.y, v1.y), v2.y),
                                  fminf(fminf(v0.z, v1.z), v2.z));
    const float3 hi = make_float3(fmaxf(fmaxf(v0.x, v1.x), v2.x), fmaxf(fmaxf(v0.y, v1.y), v2.y),
                                  fmaxf(fmaxf(v0.z, v1.z), v2.z));
    const float2 ix = unpack2(r.idir2[0]), iy = unpack2(r.idir2[1]), iz = unpack2(r.idir2[2]);
    const float2 nx = unpack2(r.noid2[0]), ny = unpack2(r.noid2[1]), nz = unpack2(r.noid2[2]);
    const float lx = fmaf(lo.x, ix.x, nx.x), hx = fmaf(hi.x, ix.x, nx.x);
    const float ly = fmaf(lo.y, iy.x, ny.x), hy = fmaf(hi.y, iy.x, ny.x);
    const float lz = fmaf(lo.z, iz.x, nz.x), hz = fmaf(hi.z, iz.x, nz.x);
    const float tn = max3(fminf(lx, hx), fminf(ly, hy), fmaxf(fminf(lz, hz), 0.0f));
    const float tf = min3(fmaxf(lx, hx), fmaxf(ly, hy), fminf(fmaxf(lz, hz), INFINITY));
    return tn <= tf * 1.00000024f;
}

// Triangle list of the 8 x 4-pixel tile (tx, ty) (one warp of the trace),
// kept in the tile's own G-buffer depth storage until the warp overwrites it:
// the tile's rows of elements (ew 32-bit words each: 4 in FP32, 2 in FP16)
// one after the other; word 0 = number of entries, words 1.. = entries
// (leaf index | kThinBit for a triangle of (near) zero area).
constexpr uint32_t kThinBit = 0x80000000u;
constexpr int kRasterTileW = 8, kRasterTileH = 4;
constexpr int kMaxBin = 48;             // longer lists: the tile is traversed

struct TileStore {
    uint32_t* base;   // the G-buffer depth storage as words
    int W, H, ew;
};

__device__ __forceinline__ int tile_row_words(const TileStore& s, int tx) { return min(kRasterTileW, s.W - kRasterTileW * tx) * s.ew; }
__device__ __forceinline__ int tile_capacity(const TileStore& s, int tx, int ty) {
    return min(kRasterTileH, s.H - kRasterTileH * ty) * tile_row_words(s, tx) - 1;
}
// word k of the tile (the tile's origin must lie inside the image)
__device__ __forceinline__ uint32_t* tile_word(const TileStore& s, int tx, int ty, int k) {
    const int wpr = tile_row_words(s, tx);
    const long long i = ((long long)(kRasterTileH * ty + k / wpr) * s.W + kRasterTileW * tx) * s.ew + k % wpr;
    return s.base + dbg_index(i, (long long)s.W * s.H * s.ew, kSiteRasterList);
}

// Pixel of a thread: each warp covers an 8x4 tile; a 128-thread block
// covers 16x8 pixels.
__device__ __forceinline__ int2 thread_pixel() {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    return make_int2(blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7),
                     blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3));
}

// kStats: also count rays, node visits and triangle tests per ray type into
// stats[0..8] = rays {primary, shadow, AO}, visits {..}, tests {..}.
// One pixel of the trace: primary ray -> G-buffer; unless kPrimaryOnly,
// the shadow and AO rays -> bitmask and count.
// kSel: shadow rays only for the pixels the lights' shadow maps cannot
// decide (smap_classify); ray_mask (optional) receives bit l = light l's
// ray was called for.
// kRaster: the primary hit is the closest among the triangles binned to the
// warp's tile (raster_device.cuh), read from the tile's G-buffer storage
// before the warp overwrites it; a tile whose list is too long or did not fit
// is traversed.  kWarps: warps per block (the warp's 32 lanes must cover one
// 8 x 4-pixel tile).  kShadowStart: shadow rays start at their segment's
// start cell (else at the root).
template <bool kHalf, bool kStats, bool kPrimaryOnly, bool kSel = false, bool kRaster = false, int kWarps = 4,
          bool kShadowStart = true>
__device__ __forceinline__ void trace_pixel(const SceneView& sc, const TraceConsts& k, int2 px, void* gbuf_dn,
                                            uint32_t* gbuf_mesh, uint8_t* mask_out, uint8_t* ao_out,
                                            unsigned long long* stats, const SmapSet* sel = nullptr,
                                            uint8_t* ray_mask = nullptr) {
    const int W = k.cam.width, H = k.cam.height;
    int n_list = -1;             // kRaster: entries of the warp's tile list to test (-1: traverse)
    const uint32_t* list = nullptr;
    if constexpr (kRaster) {
        // the whole warp copies its tile's list to shared memory before any
        // lane writes its pixel (which holds part of the list)
        __shared__ uint32_t s_list[kWarps][kMaxBin];   // kWarps warps per block
        const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
        list = s_list[wib];
        const int tx = px.x / kRasterTileW, ty = px.y / kRasterTileH;
        const TileStore ts{reinterpret_cast<uint32_t*>(gbuf_dn), W, H, kHalf ? 2 : 4};
        if (kRasterTileW * tx < W && kRasterTileH * ty < H) {
            const uint32_t n = *tile_word(ts, tx, ty, 0);
            if (n <= (uint32_t)min(kMaxBin, tile_capacity(ts, tx, ty))) {
                n_list = (int)n;
                for (int i = lane; i < n_list; i += 32) s_list[wib][i] = *tile_word(ts, tx, ty, i + 1);
            }
        }
        __syncwarp();
    }
    if (px.x >= W || px.y >= H) return;
    const size_t pix = (size_t)px.y * W + px.x;
    // primary ray through the pixel centre; its parameter is the linear depth
    const float3 eye = make_float3(k.cam.pos[0], k.cam.pos[1], k.cam.pos[2]);
    const float3 fw = make_float3(k.cam.forward[0], k.cam.forward[1], k.cam.forward[2]);
    const float3 D = primary_dir(k.cam, px.x, px.y);
    const Ray pr = make_ray(eye, D);
    float tp = INFINITY;
    float3 bary;
    Work wp, ws, wa;
    uint32_t n_sh = 0, n_ao = 0;
    int leaf = -1;
    if (kRaster && n_list >= 0) {
        // closest hit among the tile's list: smallest (t, original index), as
        // the traversal's closest hit
        if (kStats) wp.tests += (uint32_t)n_list;   // each entry: one triangle test
        uint32_t best_o = 0xFFFFFFFFu;
        for (int j = 0; j < n_list; ++j) {
            const uint32_t e = list[j];
            const int lf = (int)(e & ~kThinBit);
            if (lf >= sc.n_tris) continue;
            const float4* tr = sc.tris + 3 * lf;
            const float4 p0 = __ldg(tr), p1 = __ldg(tr + 1), p2 = __ldg(tr + 2);
            const float3 v0 = f3(p0), v1 = f3(p1), v2 = f3(p2);
            if ((e & kThinBit) && !leaf_box_hit(pr, v0, v1, v2)) continue;
            float t;
            float3 b;
            if (!hit_triangle(pr, v0, v1, v2, 0.0f, INFINITY, t, b)) continue;
            const uint32_t orig = __float_as_uint(p0.w);
            if (t < tp || (t == tp && orig < best_o)) {
                tp = t;
                best_o = orig;
                bary = b;
                leaf = lf;
            }
        }
    } else {
        leaf = traverse<false, kStats>(sc, pr, 0.0f, tp, bary, -1, &wp);
    }
    if (kStats) {
        atomicAdd(stats + 0, 1ull);
        atomicAdd(stats + 3, (unsigned long long)wp.visits);
        atomicAdd(stats + 6, (unsigned long long)wp.tests);
    }
    if (leaf < 0) {
        if (kHalf) {
            reinterpret_cast<uint2*>(gbuf_dn)[pix] = pack_gbuf16(INFINITY, make_float3(0.f, 0.f, 0.f));
        } else {
            reinterpret_cast<float4*>(gbuf_dn)[pix] = make_float4(INFINITY, 0.f, 0.f, 0.f);
        }
        gbuf_mesh[pix] = DHR_BACKGROUND;
        if (kPrimaryOnly) return;
        mask_out[pix] = (uint8_t)((1u << k.n_lights) - 1u);
        ao_out[pix] = (uint8_t)k.ao_spp;
        if constexpr (kSel) {
            if (ray_mask) ray_mask[pix] = 0;
        }
        return;
    }
    const float4* tr = sc.tris + 3 * leaf;
    const float4 p0 = __ldg(tr), p1 = __ldg(tr + 1), p2 = __ldg(tr + 2);
    const float3 v0 = f3(p0), v1 = f3(p1), v2 = f3(p2);
    // hit point from barycentrics (more accurate than eye + t D far away)
    const float3 X = make_float3(bary.x * v0.x + bary.y * v1.x + bary.z * v2.x,
                                 bary.x * v0.y + bary.y * v1.y + bary.z * v2.y,
                                 bary.x * v0.z + bary.y * v1.z + bary.z * v2.z);
    float3 n = unit_normal_rn(v0, v1, v2);
    if (dot(n, D) > 0.0f) n = make_float3(-n.x, -n.y, -n.z);
    const float depth = dot(sub(X, eye), fw);
    if (kHalf) {
        reinterpret_cast<uint2*>(gbuf_dn)[pix] = pack_gbuf16(depth, n);
    } else {
        reinterpret_cast<float4*>(gbuf_dn)[pix] = make_float4(depth, n.x, n.y, n.z);
    }
    gbuf_mesh[pix] = __float_as_uint(p1.w);
    if (kPrimaryOnly) return;

    const float3 o = surface_origin(X, n, v0, v1, v2);
    // shadow rays: one per light, direction jittered inside the light's cone
    uint32_t mask = 0, called = 0;
    for (uint32_t l = 0; l < k.n_lights; ++l) {
        if constexpr (kSel) {
            if (sel->m[l].S) {
                const int c = smap_classify(sel->m[l], X, n);
                if (c == kClsLit) mask |= 1u << l;
                if (c != kClsTrace) continue;
            }
            called |= 1u << l;
        }
        const float2 xy = disk_point(px.x, px.y, k.frame, k.seed, kShadowRay, l);
        const float3 d = cone_direction(k.light[l], k.tan_cone[l], xy);
        if (dot(d, n) <= 0.0f) continue;       // blocked by the surface itself
        float tm = INFINITY;
        float3 b;
        ++n_sh;
        const Ray ray = make_ray(o, d);
        if constexpr (kShadowStart) {
            int sd[kSeedSlots];
            const uint32_t sds = segment_start(sc, ray, sd);
            if (traverse<true, kStats, kSeedSlots>(sc, ray, 0.0f, tm, b, leaf, &ws, sd, sds) < 0) mask |= 1u << l;
        } else {
            if (traverse<true, kStats>(sc, ray, 0.0f, tm, b, leaf, &ws) < 0) mask |= 1u << l;
        }
    }
    mask_out[pix] = (uint8_t)mask;
    if constexpr (kSel) {
        if (ray_mask) ray_mask[pix] = (uint8_t)called;
    }
    // AO rays: cosine-weighted, a hit closer than r occludes (Eq. 2-3).  They
    // stay inside the ball of radius r around o; its box, padded far beyond
    // the rounding of the hit distance and of the hit point, bounds them.
    uint32_t unocc = 0;
    int seed[kSeedSlots];
    const float pad = 1e-5f * (k.ao_radius + fmaxf(fabsf(o.x), fmaxf(fabsf(o.y), fabsf(o.z))));
    const uint32_t seeds = k.ao_spp > 0 ? seed_start(sc, o, k.ao_radius + pad, seed) : 0u;
    for (uint32_t j = 0; j < k.ao_spp; ++j) {
        ++n_ao;
        if (seeds == 0) {   // no triangle near o
            ++unocc;
            continue;
        }
        const float2 xy = disk_point(px.x, px.y, k.frame, k.seed, kAoRay, j);
        const float3 d = ao_direction(n, xy);
        float tm = k.ao_radius;
        float3 b;
        if (traverse<true, kStats, kSeedSlots>(sc, make_ray(o, d), 0.0f, tm, b, leaf, &wa, seed, seeds) < 0) ++unocc;
    }
    ao_out[pix] = (uint8_t)unocc;
    if (kStats) {
        atomicAdd(stats + 1, (unsigned long long)n_sh);
        atomicAdd(stats + 2, (unsigned long long)n_ao);
        atomicAdd(stats + 4, (unsigned long long)ws.visits);
        atomicAdd(stats + 5, (unsigned long long)wa.visits);
        atomicAdd(stats + 7, (unsigned long long)ws.tests);
        atomicAdd(stats + 8, (unsigned long long)wa.tests);
    }
}


}  // namespace dhr
