// Device code of the modified SVGF (Section 3.3), shared by the forward
// entry points (svgf.cu) and the adjoint (svgf_adjoint.cu).
//
//  temporal_kernel: back-project each pixel into the previous frame, keep
//    the bilinear history taps consistent in mesh id, depth and normal,
//    accumulate colour and the first two moments with an exponential moving
//    average (alpha_eff = max(alpha, 1/n)), and estimate the variance:
//    from the moments when the history holds n >= 4 frames, else from a 7x7
//    window of the current frame weighted by depth and normal only (the
//    paper's modification: no luminance term in the variance estimate).
//  atrous_kernel: one edge-stopping a-trous iteration (5x5 B3-spline taps at
//    step 2^i, weights from depth, normal and luminance with a 3x3 Gaussian
//    of the variance); the first iteration's colour is the next frame's
//    colour history and the last iteration writes the outputs.
//
// Storage precision is a template parameter: FP32 keeps every buffer in
// binary32; FP16 stores the normal (octahedral), the colour history and the
// moments in binary16 and keeps depth and the variance-carrying buffer in
// binary32 (depth differences far below binary16 resolution drive w_z, and
// the variance mu2 - mu1^2 cancels); arithmetic is binary32.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

namespace dhr {

template <dhr_precision P>
struct Store;

template <>
struct Store<DHR_FP32> {
    using G = float4;
    using Col = float2;
    using Mom = float4;
    static __device__ __forceinline__ float4 g(const G* p, size_t i) { return __ldg(p + i); }
    static __device__ __forceinline__ float2 col(const Col* p, size_t i) { return __ldg(p + i); }
    static __device__ __forceinline__ void put_col(Col* p, size_t i, float2 v) { p[i] = v; }
    static __device__ __forceinline__ float4 mom(const Mom* p, size_t i) { return __ldg(p + i); }
    static __device__ __forceinline__ void put_mom(Mom* p, size_t i, float4 v) { p[i] = v; }
};

template <>
struct Store<DHR_FP16> {
    using G = uint2;
    using Col = __half2;
    using Mom = ushort4;
    static __device__ __forceinline__ float h(unsigned short u) { return __half2float(__ushort_as_half(u)); }
    static __device__ __forceinline__ unsigned short q(float f) { return __half_as_ushort(__float2half_rn(f)); }
    static __device__ __forceinline__ float4 g(const G* p, size_t i) { return unpack_gbuf16(__ldg(p + i)); }
    static __device__ __forceinline__ float2 col(const Col* p, size_t i) { return __half22float2(p[i]); }
    static __device__ __forceinline__ void put_col(Col* p, size_t i, float2 v) { p[i] = __float22half2_rn(v); }
    static __device__ __forceinline__ float4 mom(const Mom* p, size_t i) {
        const ushort4 u = __ldg(p + i);
        return make_float4(h(u.x), h(u.y), h(u.z), h(u.w));
    }
    static __device__ __forceinline__ void put_mom(Mom* p, size_t i, float4 v) {
        p[i] = make_ushort4(q(v.x), q(v.y), q(v.z), q(v.w));
    }
};

struct SvgfConsts {
    int W, H;
    float alpha, sigma_z, sigma_n, sigma_l, eps_z, eps_l;
    float inv_spp;
    int fixed_alpha, wl_in_atrous;
    int sigma_n_int;    // sigma_n when it is an integer in 1..1024, else 0
};

__device__ __forceinline__ bool is_fg(float z) { return z < INFINITY; }

// max(0, c)^sigma_n with 0^0 = 1.  Integer exponents up to 1024 (the usual
// case, e.g. 128) use repeated squaring: a few multiplies and relative error
// ~1e-6, where exp2(sigma_n log2 c) would amplify the log2 error sigma_n-fold.
__device__ __forceinline__ float pow_normal(float c, float sigma_n, int int_exp) {
    if (sigma_n == 0.0f) return 1.0f;
    c = fmaxf(c, 0.0f);
    if (int_exp > 0) {
        float r = 1.0f, b = c;
        for (int e = int_exp; e; e >>= 1) {
            if (e & 1) r *= b;
            b *= b;
        }
        return r;
    }
    return c > 0.0f ? exp2f(sigma_n * log2f(c)) : 0.0f;
}

__device__ __forceinline__ float w_depth(float zp, float zq, float2 g, float ox, float oy, float sz, float ez) {
    return __expf(-fabsf(zp - zq) / (sz * fabsf(fmaf(g.x, ox, g.y * oy)) + ez));
}

// per-axis one-sided depth difference of smaller magnitude (0 if none)
template <class S>
__device__ __forceinline__ float2 depth_grad(const typename S::G* g, int W, int H, int x, int y, float zp) {
    float r[2];
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const int xp = x + (ax == 0), yp = y + (ax == 1), xm = x - (ax == 0), ym = y - (ax == 1);
        bool hp = false, hm = false;
        float dp = 0.f, dm = 0.f;
        if (xp < W && yp < H) {
            const float z = S::g(g, (size_t)yp * W + xp).x;
            if (is_fg(z)) { dp = z - zp; hp = true; }
        }
        if (xm >= 0 && ym >= 0) {
            const float z = S::g(g, (size_t)ym * W + xm).x;
            if (is_fg(z)) { dm = zp - z; hm = true; }
        }
        r[ax] = (hp && hm) ? (fabsf(dm) < fabsf(dp) ? dm : dp) : (hp ? dp : (hm ? dm : 0.f));
    }
    return make_float2(r[0], r[1]);
}

__device__ __forceinline__ float2 noisy(const uint8_t* mask, const uint8_t* ao, size_t i, float inv_spp) {
    return make_float2((float)__ldg(ao + i) * inv_spp, (__ldg(mask + i) & 1u) ? 1.0f : 0.0f);
}

// noisy signals of the current frame: from the 8-bit trace outputs
// (AO = N_unoccluded / N, Eq. 3; shadow = bit 0 of the visibility mask) ...
struct SigCounts {
    const uint8_t* mask;
    const uint8_t* ao;
    float inv_spp;
    __device__ __forceinline__ float2 operator()(size_t i) const { return noisy(mask, ao, i, inv_spp); }
};

// ... or real-valued planes [2][H][W] (the differentiable form)
struct SigPlanar {
    const float* s;
    size_t plane;
    __device__ __forceinline__ float2 operator()(size_t i) const {
        return make_float2(__ldg(s + i), __ldg(s + plane + i));
    }
};

// Back-projection into the previous frame: the binary32 operation sequence
// below (each step rounded once, no contraction) decides which history taps
// are valid; it is the specification shared with the CPU oracle.  Depth
// consistency: |z_prev(q) - z'| <= 0.01 z' + 2 max(|dz/dx|, |dz/dy|).
struct Reproj {
    int x0, y0;
    float w[4];
    int ok;          // bit k: tap k valid (00, 10, 01, 11)
    float sumw;
};

template <class S>
__device__ __forceinline__ bool reproject(const dhr_camera& c, const dhr_camera& p, int W, int H, int x, int y,
                                          float4 znp, uint32_t mp, float slope, const typename S::G* g_prev,
                                          const uint32_t* mesh_prev, Reproj& r) {
    const float Wf = (float)W, Hf = (float)H;
    const float aspect = __fdiv_rn(Wf, Hf);
    const float fx = __fadd_rn((float)x, 0.5f), fy = __fadd_rn((float)y, 0.5f);
    const float qx = __fdiv_rn(__fmul_rn(2.0f, fx), Wf), qy = __fdiv_rn(__fmul_rn(2.0f, fy), Hf);
    const float ndx = __fsub_rn(qx, 1.0f), ndy = __fsub_rn(1.0f, qy);
    const float sx = __fmul_rn(__fmul_rn(ndx, c.tan_half_fov_y), aspect);
    const float sy = __fmul_rn(ndy, c.tan_half_fov_y);
    float rr[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float D = __fadd_rn(__fadd_rn(c.forward[k], __fmul_rn(sx, c.right[k])), __fmul_rn(sy, c.up[k]));
        const float X = __fadd_rn(c.pos[k], __fmul_rn(znp.x, D));
        rr[k] = __fsub_rn(X, p.pos[k]);
    }
    const float zp = __fadd_rn(__fadd_rn(__fmul_rn(rr[0], p.forward[0]), __fmul_rn(rr[1], p.forward[1])),
                               __fmul_rn(rr[2], p.forward[2]));
    const float rx = __fadd_rn(__fadd_rn(__fmul_rn(rr[0], p.right[0]), __fmul_rn(rr[1], p.right[1])),
                               __fmul_rn(rr[2], p.right[2]));
    const float ry = __fadd_rn(__fadd_rn(__fmul_rn(rr[0], p.up[0]), __fmul_rn(rr[1], p.up[1])),
                               __fmul_rn(rr[2], p.up[2]));
    if (!(zp > 0.0f)) return false;
    const float zt = __fmul_rn(zp, p.tan_half_fov_y);
    const float zta = __fmul_rn(zt, aspect);
    const float su = __fdiv_rn(rx, zta), sv = __fdiv_rn(ry, zt);
    const float pxc = __fmul_rn(__fmul_rn(__fadd_rn(su, 1.0f), 0.5f), Wf);
    const float pyc = __fmul_rn(__fmul_rn(__fsub_rn(1.0f, sv), 0.5f), Hf);
    const float gx = __fsub_rn(pxc, 0.5f), gy = __fsub_rn(pyc, 0.5f);
    if (!(gx > -1.0f && gx < Wf && gy > -1.0f && gy < Hf)) return false;
    const float x0f = floorf(gx), y0f = floorf(gy);
    const float ax = __fsub_rn(gx, x0f), ay = __fsub_rn(gy, y0f);
    const float bx = __fsub_rn(1.0f, ax), by = __fsub_rn(1.0f, ay);
    r.w[0] = __fmul_rn(bx, by);
    r.w[1] = __fmul_rn(ax, by);
    r.w[2] = __fmul_rn(bx, ay);
    r.w[3] = __fmul_rn(ax, ay);
    r.x0 = (int)x0f;
    r.y0 = (int)y0f;
    // projected depths agree within 1 % plus two pixels of the local depth slope
    const float zlim = __fadd_rn(__fmul_rn(0.01f, zp), __fmul_rn(2.0f, slope));
    float sumw = 0.0f;
    int ok = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int qx2 = r.x0 + (k & 1), qy2 = r.y0 + (k >> 1);
        if (qx2 < 0 || qy2 < 0 || qx2 >= W || qy2 >= H) continue;
        const size_t q = (size_t)qy2 * W + qx2;
        if (__ldg(mesh_prev + q) != mp) continue;
        const float4 gq = S::g(g_prev, q);
        if (!(fabsf(__fsub_rn(gq.x, zp)) <= zlim)) continue;
        const float nd = __fadd_rn(__fadd_rn(__fmul_rn(znp.y, gq.y), __fmul_rn(znp.z, gq.z)), __fmul_rn(znp.w, gq.w));
        if (!(nd >= 0.9f)) continue;
        ok |= 1 << k;
        sumw = __fadd_rn(sumw, r.w[k]);
    }
    r.ok = ok;
    r.sumw = sumw;
    return sumw >= 1e-4f;
}

constexpr unsigned kFull = 0xffffffffu;
constexpr float kLog2e = 1.4426950408889634f;

// Background pixels carry variance -1 in the illum buffers (a sentinel
// that lets the a-trous passes test membership from the buffer they read).
__device__ __forceinline__ bool fg_var(float v) { return v >= 0.0f; }

// Temporal step for the 32x8 tile at (bx0, by0), run by a 32x8 block.
template <dhr_precision P, class Sig>
__device__ __forceinline__ void temporal_tile(
    const SvgfConsts& k, const dhr_camera& cam, const dhr_camera& cam_prev, const typename Store<P>::G* g_cur,
    const uint32_t* mesh_cur, const typename Store<P>::G* g_prev, const uint32_t* mesh_prev,
    const Sig& sig, const typename Store<P>::Col* col_hist,
    const typename Store<P>::Mom* mom_in, const uint8_t* hist_in, typename Store<P>::Mom* mom_out,
    uint8_t* hist_out, float4* illum, int bx0, int by0) {
    using S = Store<P>;
    // one warp = 32 consecutive pixels of a row; every lane stays to the end
    // because the short-history estimate below is computed by the whole warp
    const int x = bx0 + threadIdx.x, y = by0 + threadIdx.y;
    const int lane = threadIdx.x & 31;
    const bool inside = x < k.W && y < k.H;
    const size_t p = inside ? (size_t)y * k.W + x : 0;
    float4 zn = make_float4(INFINITY, 0.f, 0.f, 0.f);
    if (inside) zn = S::g(g_cur, p);
    const bool fg = inside && is_fg(zn.x);
    int n = 1;
    float2 gz = make_float2(0.f, 0.f);
    if (fg) {
        const float2 s = sig(p);
        float2 ch = make_float2(0.f, 0.f);
        float4 mh = make_float4(0.f, 0.f, 0.f, 0.f);
        bool valid = false;
        Reproj r;
        gz = depth_grad<S>(g_cur, k.W, k.H, x, y, zn.x);
        const float slope = fmaxf(fabsf(gz.x), fabsf(gz.y));
        if (g_prev &&
            reproject<S>(cam, cam_prev, k.W, k.H, x, y, zn, __ldg(mesh_cur + p), slope, g_prev, mesh_prev, r)) {
            // weighted mean of the valid taps as (sum w v) / (sum w), summed in the
            // same order as sum w so that a constant history stays exactly constant
            valid = true;
            int hmin = 255;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (!(r.ok & (1 << t))) continue;
                const size_t q = (size_t)(r.y0 + (t >> 1)) * k.W + (r.x0 + (t & 1));
                const float w = r.w[t];
                const float2 c = S::col(col_hist, q);
                const float4 m = S::mom(mom_in, q);
                ch.x = fmaf(w, c.x, ch.x);
                ch.y = fmaf(w, c.y, ch.y);
                mh.x = fmaf(w, m.x, mh.x);
                mh.y = fmaf(w, m.y, mh.y);
                mh.z = fmaf(w, m.z, mh.z);
                mh.w = fmaf(w, m.w, mh.w);
                hmin = min(hmin, (int)__ldg(hist_in + q));
            }
            ch = make_float2(ch.x / r.sumw, ch.y / r.sumw);
            mh = make_float4(mh.x / r.sumw, mh.y / r.sumw, mh.z / r.sumw, mh.w / r.sumw);
            n = min(hmin + 1, 255);
        }
        const float a = valid ? (k.fixed_alpha ? k.alpha : fmaxf(k.alpha, 1.0f / (float)n)) : 1.0f;
        // exponential moving average written h + a (s - h)
        const float2 c = make_float2(fmaf(a, s.x - ch.x, ch.x), fmaf(a, s.y - ch.y, ch.y));
        const float4 m = make_float4(fmaf(a, s.x - mh.x, mh.x), fmaf(a, s.y - mh.y, mh.y),
                                     fmaf(a, s.x * s.x - mh.z, mh.z), fmaf(a, s.y * s.y - mh.w, mh.w));
        S::put_mom(mom_out, p, m);
        hist_out[p] = (uint8_t)n;
        if (n >= 4)
            illum[p] = make_float4(c.x, c.y, fmaxf(0.f, m.z - m.x * m.x), fmaxf(0.f, m.w - m.y * m.y));
    } else if (inside) {
        illum[p] = make_float4(1.f, 1.f, -1.f, -1.f);
        S::put_mom(mom_out, p, make_float4(1.f, 1.f, 1.f, 1.f));
        hist_out[p] = 0;
    }
    // short history (n < 4): 7x7 spatial estimate of the current frame's
    // signal weighted by depth and normal only.  The lanes that need it are
    // served one after another by the whole warp: lane l takes taps l and
    // l + 32 of the 49, then the sums are reduced across the warp.
    const bool need = fg && n < 4;
    unsigned todo = __ballot_sync(kFull, need);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int px = __shfl_sync(kFull, x, src), py = __shfl_sync(kFull, y, src);
        const float zp = __shfl_sync(kFull, zn.x, src);
        const float nx = __shfl_sync(kFull, zn.y, src), ny = __shfl_sync(kFull, zn.z, src),
                    nz = __shfl_sync(kFull, zn.w, src);
        const float gx = __shfl_sync(kFull, gz.x, src), gy = __shfl_sync(kFull, gz.y, src);
        float sw = 0.f, a1 = 0.f, b1 = 0.f, a2 = 0.f, b2 = 0.f;
        for (int t = lane; t < 49; t += 32) {
            const int dx = t % 7 - 3, dy = t / 7 - 3;
            const int qx = px + dx, qy = py + dy;
            if (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H) continue;
            const size_t q = (size_t)qy * k.W + qx;
            const float4 zq = S::g(g_cur, q);
            if (!is_fg(zq.x)) continue;
            float w = 1.0f;
            if (dx || dy)
                w = w_depth(zp, zq.x, make_float2(gx, gy), (float)-dx, (float)-dy, k.sigma_z, k.eps_z) *
                    pow_normal(nx * zq.y + ny * zq.z + nz * zq.w, k.sigma_n, k.sigma_n_int);
            const float2 sq = sig(q);
            sw += w;
            a1 = fmaf(w, sq.x, a1);
            b1 = fmaf(w, sq.y, b1);
            a2 = fmaf(w, sq.x * sq.x, a2);
            b2 = fmaf(w, sq.y * sq.y, b2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sw += __shfl_xor_sync(kFull, sw, o);
            a1 += __shfl_xor_sync(kFull, a1, o);
            b1 += __shfl_xor_sync(kFull, b1, o);
            a2 += __shfl_xor_sync(kFull, a2, o);
            b2 += __shfl_xor_sync(kFull, b2, o);
        }
        if (lane == src) {
            const float m1x = a1 / sw, m1y = b1 / sw;
            illum[p] = make_float4(m1x, m1y, fmaxf(0.f, a2 / sw - m1x * m1x), fmaxf(0.f, b2 / sw - m1y * m1y));
        }
    }
}

template <dhr_precision P, class Sig>
__global__ void __launch_bounds__(256) temporal_kernel(
    SvgfConsts k, dhr_camera cam, dhr_camera cam_prev, const typename Store<P>::G* g_cur,
    const uint32_t* mesh_cur, const typename Store<P>::G* g_prev, const uint32_t* mesh_prev,
    Sig sig, const typename Store<P>::Col* col_hist,
    const typename Store<P>::Mom* mom_in, const uint8_t* hist_in, typename Store<P>::Mom* mom_out,
    uint8_t* hist_out, float4* illum) {
    temporal_tile<P, Sig>(k, cam, cam_prev, g_cur, mesh_cur, g_prev, mesh_prev, sig, col_hist, mom_in, hist_in,
                          mom_out, hist_out, illum, blockIdx.x * 32, blockIdx.y * 8);
}

// max(0, c)^sigma_n for the a-trous taps: 2^kNsq by kNsq squarings, or the
// generic path (kNsq < 0)
template <int kNsq>
__device__ __forceinline__ float pow_n(float c, float sigma_n, int sigma_n_int) {
    if (kNsq >= 0) {
        float r = fmaxf(c, 0.0f);
#pragma unroll
        for (int i = 0; i < kNsq; ++i) r *= r;
        return r;
    }
    return pow_normal(c, sigma_n, sigma_n_int);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Acc {
    float sw0, sw1, sc0, sc1, sv0, sv1;
};

// The 24 non-centre taps of one a-trous iteration.  Background taps (depth
// +inf, variance sentinel -1) get weight 0 without a branch.
template <class S, int kNsq, bool kCheck>
__device__ __forceinline__ void atrous_taps(const SvgfConsts& k, int step, int x, int y, float4 zn, float4 cp,
                                            float il0, float il1, const float (&rz)[13],
                                            const typename S::G* g, const float4* in, Acc& a) {
    const float h5[5] = {1.f / 16, 1.f / 4, 3.f / 8, 1.f / 4, 1.f / 16};
#pragma unroll
    for (int j = -2; j <= 2; ++j) {
        const int qy = y + j * step;
        if (kCheck && (qy < 0 || qy >= k.H)) continue;
#pragma unroll
        for (int i = -2; i <= 2; ++i) {
            if (i == 0 && j == 0) continue;
            const int qx = x + i * step;
            if (kCheck && (qx < 0 || qx >= k.W)) continue;
            const int q = qy * k.W + qx;
            const float4 cq = __ldg(in + q);
            const float4 zq = S::g(g, q);
            const int t = (j < 0 || (j == 0 && i < 0)) ? (j + 2) * 5 + (i + 2) : (2 - j) * 5 + (2 - i);
            const float ez = fabsf(zn.x - zq.x) * rz[t];
            float kw = h5[i + 2] * h5[j + 2] *
                       pow_n<kNsq>(zn.y * zq.y + zn.z * zq.z + zn.w * zq.w, k.sigma_n, k.sigma_n_int);
            kw = fg_var(cq.z) ? kw : 0.0f;
            float w0 = kw * ex2_approx(-fmaf(fabsf(cp.x - cq.x), il0, ez));
            float w1 = kw * ex2_approx(-fmaf(fabsf(cp.y - cq.y), il1, ez));
            w0 = fg_var(cq.z) ? w0 : 0.0f;    // NaN-safe for whatever a background pixel holds
            w1 = fg_var(cq.z) ? w1 : 0.0f;
            a.sw0 += w0;
            a.sw1 += w1;
            a.sc0 = fmaf(w0, cq.x, a.sc0);
            a.sc1 = fmaf(w1, cq.y, a.sc1);
            a.sv0 = fmaf(w0 * w0, cq.z, a.sv0);
            a.sv1 = fmaf(w1 * w1, cq.w, a.sv1);
        }
    }
}

// one a-trous iteration; kMode 0: write illum_out; 1: also colour history;
// 2: last iteration, write the two output planes only.  kNsq >= 0: sigma_n
// is 2^kNsq.
template <dhr_precision P, int kMode, int kNsq>
__device__ __forceinline__ void atrous_tile(const SvgfConsts& k, int step, const typename Store<P>::G* g,
                                            const float4* in, float4* out, typename Store<P>::Col* col_hist,
                                            float* ao_out, float* sh_out, int bx0, int by0) {
    using S = Store<P>;
    const int x = bx0 + threadIdx.x, y = by0 + threadIdx.y;
    if (x >= k.W || y >= k.H) return;
    const int p = y * k.W + x;
    const float4 cp = __ldg(in + p);
    if (!fg_var(cp.z)) {
        if (kMode == 2) {
            ao_out[p] = 1.f;
            sh_out[p] = 1.f;
        } else {
            out[p] = make_float4(1.f, 1.f, -1.f, -1.f);
            if (kMode == 1) S::put_col(col_hist, p, make_float2(1.f, 1.f));
        }
        return;
    }
    const float4 zn = S::g(g, p);
    // 3x3 Gaussian of the variance, renormalised over foreground taps
    float gv0 = 0.f, gv1 = 0.f, gw = 0.f;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int qx = x + dx, qy = y + dy;
            if (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H) continue;
            const float4 v = __ldg(in + (qy * k.W + qx));
            if (!fg_var(v.z)) continue;
            const float kk = (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f);
            gw += kk;
            gv0 = fmaf(kk, v.z, gv0);
            gv1 = fmaf(kk, v.w, gv1);
        }
    }
    // luminance terms folded with log2(e): w_l = 2^(-|dc| il)
    const float il0 = k.wl_in_atrous ? kLog2e / (k.sigma_l * sqrtf(gv0 / gw) + k.eps_l) : 0.f;
    const float il1 = k.wl_in_atrous ? kLog2e / (k.sigma_l * sqrtf(gv1 / gw) + k.eps_l) : 0.f;
    // depth terms: log2(e) / (sigma_z |grad z . (p - q)| + eps_z) for the 12
    // offset directions (i, j) ~ (-i, -j) of the 5x5 footprint
    const float2 gz = depth_grad<S>(g, k.W, k.H, x, y, zn.x);
    const float sg = k.sigma_z * (float)step;
    float rz[13];
#pragma unroll
    for (int t = 0; t < 13; ++t) {
        const int i = t % 5 - 2, j = t / 5 - 2;      // t = 0..12 covers j < 0, and j = 0, i < 0 (t = 10, 11) + centre (12)
        rz[t] = __fdividef(kLog2e, fmaf(sg, fabsf(fmaf(gz.x, (float)i, gz.y * (float)j)), k.eps_z));
    }
    const float kc = 0.375f * 0.375f;
    Acc acc;
    acc.sw0 = kc;
    acc.sw1 = kc;
    acc.sc0 = kc * cp.x;
    acc.sc1 = kc * cp.y;
    acc.sv0 = kc * kc * cp.z;
    acc.sv1 = kc * kc * cp.w;
    // blocks whose 5x5 footprint lies inside the image skip the bounds tests
    const bool interior = bx0 - 2 * step >= 0 && by0 - 2 * step >= 0 &&
                          bx0 + (int)blockDim.x - 1 + 2 * step < k.W && by0 + (int)blockDim.y - 1 + 2 * step < k.H;
    if (interior)
        atrous_taps<S, kNsq, false>(k, step, x, y, zn, cp, il0, il1, rz, g, in, acc);
    else
        atrous_taps<S, kNsq, true>(k, step, x, y, zn, cp, il0, il1, rz, g, in, acc);
    const float sw0 = acc.sw0, sw1 = acc.sw1, sc0 = acc.sc0, sc1 = acc.sc1, sv0 = acc.sv0, sv1 = acc.sv1;
    // (sum w c) / (sum w): a constant neighbourhood stays exactly constant
    const float c0 = sc0 / sw0, c1 = sc1 / sw1;
    if (kMode == 2) {
        ao_out[p] = c0;
        sh_out[p] = c1;
    } else {
        out[p] = make_float4(c0, c1, sv0 / (sw0 * sw0), sv1 / (sw1 * sw1));
        if (kMode == 1) S::put_col(col_hist, p, make_float2(c0, c1));
    }
}

template <dhr_precision P, int kMode, int kNsq>
__global__ void __launch_bounds__(256) atrous_kernel(SvgfConsts k, int step, const typename Store<P>::G* g,
                                                     const float4* in, float4* out,
                                                     typename Store<P>::Col* col_hist, float* ao_out,
                                                     float* sh_out) {
    atrous_tile<P, kMode, kNsq>(k, step, g, in, out, col_hist, ao_out, sh_out, blockIdx.x * blockDim.x,
                                blockIdx.y * blockDim.y);
}

// levels == 0: the temporal colour is the output and the colour history
template <dhr_precision P>
__global__ void passthrough_kernel(int n, const float4* illum, typename Store<P>::Col* col_hist, float* ao_out,
                                   float* sh_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = illum[i];
    Store<P>::put_col(col_hist, i, make_float2(v.x, v.y));
    ao_out[i] = v.x;
    sh_out[i] = v.y;
}


inline SvgfConsts make_consts(int W, int H, const dhr_svgf_params* prm) {
    SvgfConsts k;
    k.W = W;
    k.H = H;
    k.alpha = prm->alpha;
    k.sigma_z = prm->sigma_z;
    k.sigma_n = prm->sigma_n;
    k.sigma_l = prm->sigma_l;
    k.eps_z = prm->eps_z;
    k.eps_l = prm->eps_l;
    k.inv_spp = 1.0f / (float)prm->ao_spp;
    k.fixed_alpha = (int)prm->fixed_alpha;
    k.wl_in_atrous = (int)prm->wl_in_atrous;
    k.sigma_n_int = (prm->sigma_n >= 1.0f && prm->sigma_n <= 1024.0f && prm->sigma_n == floorf(prm->sigma_n))
                        ? (int)prm->sigma_n : 0;
    return k;
}

inline int atrous_nsq(const dhr_svgf_params* prm) { return prm->sigma_n == 128.0f ? 7 : -1; }

template <dhr_precision P, int kMode>
inline void launch_atrous_mode(int nsq, dim3 grid, dim3 blk, cudaStream_t st, const SvgfConsts& k, int step,
                               const typename Store<P>::G* g, const float4* in, float4* out,
                               typename Store<P>::Col* col, float* ao_out, float* sh_out) {
    if (nsq == 7)
        atrous_kernel<P, kMode, 7><<<grid, blk, 0, st>>>(k, step, g, in, out, col, ao_out, sh_out);
    else
        atrous_kernel<P, kMode, -1><<<grid, blk, 0, st>>>(k, step, g, in, out, col, ao_out, sh_out);
}

template <dhr_precision P>
inline dhr_status launch_atrous(int mode, int nsq, dim3 grid, dim3 blk, cudaStream_t st, const SvgfConsts& k,
                                int step, const typename Store<P>::G* g, const float4* in, float4* out,
                                typename Store<P>::Col* col, float* ao_out, float* sh_out) {
    if (mode == 2)
        launch_atrous_mode<P, 2>(nsq, grid, blk, st, k, step, g, in, nullptr, nullptr, ao_out, sh_out);
    else if (mode == 1)
        launch_atrous_mode<P, 1>(nsq, grid, blk, st, k, step, g, in, out, col, nullptr, nullptr);
    else
        launch_atrous_mode<P, 0>(nsq, grid, blk, st, k, step, g, in, out, nullptr, nullptr, nullptr);
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}

}  // namespace dhr
