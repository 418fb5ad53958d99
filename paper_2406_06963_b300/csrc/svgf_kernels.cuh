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
// binary32; the 16-bit form (DHR_FP16) stores the normal (octahedral) and
// the first moments in 16 bits and keeps depth, the colour history and the
// variances in binary32; arithmetic is binary32.  Why those in 32 bits:
// depth differences far below 16-bit resolution drive w_z; a moving average
// stored in 16 bits stops moving once alpha |s - h| is below half a step
// (binary16: up to 2^-12 / alpha = 1.2e-3 away from its input near 1), and
// the colour history feeds the output directly; mu2 - mu1^2 cancels, so the
// second moment is kept as the variance itself.
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
    static __device__ __forceinline__ void put_mom(Mom* p, size_t i, float4 v, float2) { p[i] = v; }
};

// 16-bit moments record, 12 bytes: mu1 (AO, shadow) as two 16-bit
// unsigned-normalised values q / 65535 (the signals and their means lie in
// [0, 1]; every 8-bit AO fraction k / 255 is exact, 65535 = 255 x 257, and a
// step of 1.5e-5 leaves a moving average at most 3.8e-5 from a constant
// input, a variance floor far below what the luminance weight resolves),
// then the two variances mu2 - mu1^2 in binary32.
__device__ __forceinline__ uint32_t unorm16(float v) {
    return (uint32_t)__float2uint_rn(fminf(fmaxf(v, 0.0f), 1.0f) * 65535.0f);
}

struct Mom16 {
    uint32_t mu1;        // AO in bits 0-15, shadow in bits 16-31
    float var_ao, var_sh;
};
static_assert(sizeof(Mom16) == 12, "16-bit moments record must stay 12 bytes");

template <>
struct Store<DHR_FP16> {
    using G = uint2;
    using Col = float2;
    using Mom = Mom16;
    static __device__ __forceinline__ float4 g(const G* p, size_t i) { return unpack_gbuf16(__ldg(p + i)); }
    static __device__ __forceinline__ float2 col(const Col* p, size_t i) { return __ldg(p + i); }
    static __device__ __forceinline__ void put_col(Col* p, size_t i, float2 v) { p[i] = v; }
    // (mu1, mu2) with mu2 rebuilt from the stored mu1 and variance, so that
    // mu2 - mu1^2 gives back the stored variance
    static __device__ __forceinline__ float4 mom(const Mom* p, size_t i) {
        const uint32_t u = __ldg(&p[i].mu1);
        const float mx = (float)(u & 0xFFFFu) * (1.0f / 65535.0f), my = (float)(u >> 16) * (1.0f / 65535.0f);
        const float va = __ldg(&p[i].var_ao), vs = __ldg(&p[i].var_sh);
        return make_float4(mx, my, fmaf(mx, mx, va), fmaf(my, my, vs));
    }
    static __device__ __forceinline__ void put_mom(Mom* p, size_t i, float4 v, float2) {
        p[i].mu1 = unorm16(v.x) | (unorm16(v.y) << 16);
        p[i].var_ao = fmaxf(0.f, v.z - v.x * v.x);
        p[i].var_sh = fmaxf(0.f, v.w - v.y * v.y);
    }
};

// Internal storage tag for the a-trous levels of an FP16 state: colour
// history as in FP16, the G-buffer read from a float4 copy decoded once per
// frame (instead of decoding the octahedral normal at every tap).
constexpr dhr_precision kFP16Decoded = static_cast<dhr_precision>(0x10);

template <>
struct Store<kFP16Decoded> {
    using G = float4;
    using Col = float2;
    using Mom = Mom16;
    static __device__ __forceinline__ float4 g(const G* p, size_t i) { return __ldg(p + i); }
    static __device__ __forceinline__ void put_col(Col* p, size_t i, float2 v) { p[i] = v; }
};

struct SvgfConsts {
    int W, H;
    float alpha, sigma_z, sigma_n, sigma_l, eps_z, eps_l;
    float inv_spp;
    int fixed_alpha, wl_in_atrous;
    uint32_t shadow_bit;   // light whose visibility bit is the shadow channel
};

__device__ __forceinline__ bool is_fg(float z) { return z < INFINITY; }

// Depth slope along one axis from the one-sided differences toward the two
// neighbours (minmod): the one of smaller magnitude when both have the same
// sign, 0 when their signs differ (a one-pixel ridge or valley) or one is 0;
// with one foreground neighbour its difference, with none 0.  Unlike "the
// smaller magnitude" alone it is continuous in the depths, so a rounding
// change of a depth cannot swing the slope from +d to -d.
__device__ __forceinline__ float minmod_slope(bool hp, float dp, bool hm, float dm) {
    if (hp && hm)
        return ((dp > 0.f && dm > 0.f) || (dp < 0.f && dm < 0.f)) ? (fabsf(dm) < fabsf(dp) ? dm : dp) : 0.f;
    return hp ? dp : (hm ? dm : 0.f);
}

// per-axis depth slope (minmod of the one-sided differences)
template <class S>
__device__ __forceinline__ float2 depth_grad(const typename S::G* g, int W, int H, int x, int y, float zp) {
    float r[2];
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const int xp = x + (ax == 0), yp = y + (ax == 1), xm = x - (ax == 0), ym = y - (ax == 1);
        bool hp = false, hm = false;
        float dp = 0.f, dm = 0.f;
        if (xp < W && yp < H) {
            const float z = S::g(g, dbg_index((long long)yp * W + xp, (long long)W * H, kSiteDepthGrad)).x;
            if (is_fg(z)) { dp = z - zp; hp = true; }
        }
        if (xm >= 0 && ym >= 0) {
            const float z = S::g(g, dbg_index((long long)ym * W + xm, (long long)W * H, kSiteDepthGrad)).x;
            if (is_fg(z)) { dm = zp - z; hm = true; }
        }
        r[ax] = minmod_slope(hp, dp, hm, dm);
    }
    return make_float2(r[0], r[1]);
}

__device__ __forceinline__ float2 noisy(const uint8_t* mask, const uint8_t* ao, size_t i, float inv_spp,
                                       uint32_t bit) {
    return make_float2((float)__ldg(ao + i) * inv_spp, ((__ldg(mask + i) >> bit) & 1u) ? 1.0f : 0.0f);
}

// noisy signals of the current frame: from the 8-bit trace outputs
// (AO = N_unoccluded / N, Eq. 3; shadow = bit `bit` of the visibility mask,
// one bit per light) ...
struct SigCounts {
    const uint8_t* mask;
    const uint8_t* ao;
    float inv_spp;
    uint32_t bit;
    __device__ __forceinline__ float2 operator()(size_t i) const { return noisy(mask, ao, i, inv_spp, bit); }
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
// consistency: |z_prev(q) - z'| <= 0.01 z' + 2 max(|dz/dx|, |dz/dy|), the
// slopes those of depth_grad.
struct Reproj {
    int x0, y0;
    float w[4];
    int q[4];        // tap addresses, clamped into the image
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
    // the four taps' loads are issued together (addresses clamped into the
    // image); taps outside the image are rejected afterwards
    uint32_t mq[4];
    float4 gq[4];
    bool inb[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int qx2 = r.x0 + (k & 1), qy2 = r.y0 + (k >> 1);
        inb[k] = qx2 >= 0 && qy2 >= 0 && qx2 < W && qy2 < H;
        r.q[k] = (int)dbg_index((long long)min(max(qy2, 0), H - 1) * W + min(max(qx2, 0), W - 1), (long long)W * H,
                                kSiteReproject);
        mq[k] = __ldg(mesh_prev + r.q[k]);
        gq[k] = S::g(g_prev, r.q[k]);
    }
    float sumw = 0.0f;
    int ok = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!inb[k] || mq[k] != mp) continue;
        if (!(fabsf(__fsub_rn(gq[k].x, zp)) <= zlim)) continue;
        const float nd = __fadd_rn(__fadd_rn(__fmul_rn(znp.y, gq[k].y), __fmul_rn(znp.z, gq[k].z)),
                                   __fmul_rn(znp.w, gq[k].w));
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

// 2^x and log2(x) by the hardware approximations (ftz)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x and sqrt(x) by the hardware approximations (ftz): one special-function
// instruction each, for weights and scales that need no correct rounding
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Background pixels carry variance -1 in the illum buffers (a sentinel
// that lets the a-trous passes test membership from the buffer they read).
__device__ __forceinline__ bool fg_var(float v) { return v >= 0.0f; }

// w_z w_n of the 7x7 short-history estimate for the tap at offset (dx, dy)
// from a centre of depth zp, normal np and depth gradient gz:
//   2^(-|dz| log2(e) / (sigma_z |grad z . (p - q)| + eps_z) + sigma_n log2(n.n_q))
__device__ __forceinline__ float w_spatial(const SvgfConsts& k, float zp, float3 np, float2 gz, int dx, int dy,
                                           float4 zq) {
    if (!(dx || dy)) return 1.0f;
    const float rz = kLog2e * rcp_approx(fmaf(k.sigma_z, fabsf(fmaf(gz.x, (float)-dx, gz.y * (float)-dy)), k.eps_z));
    const float ln = k.sigma_n == 0.0f
                         ? 0.0f
                         : k.sigma_n * lg2_approx(fmaxf(np.x * zq.y + np.y * zq.z + np.z * zq.w, 0.0f));
    return ex2_approx(fmaf(-fabsf(zp - zq.x), rz, ln));
}

// A warp with at least this many short-history lanes lets each of them
// compute its own 7x7 estimate; with fewer, the warp serves them one after
// another (each a single pass of the whole warp over the 49 taps).
constexpr int kShortPerLane = 8;

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
            float2 cv[4];
            float4 mv[4];
            int hv[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {       // loads first, all four taps at once
                cv[t] = S::col(col_hist, r.q[t]);
                mv[t] = S::mom(mom_in, r.q[t]);
                hv[t] = __ldg(hist_in + r.q[t]);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (!(r.ok & (1 << t))) continue;
                const float w = r.w[t];
                const float2 c = cv[t];
                const float4 m = mv[t];
                ch.x = fmaf(w, c.x, ch.x);
                ch.y = fmaf(w, c.y, ch.y);
                mh.x = fmaf(w, m.x, mh.x);
                mh.y = fmaf(w, m.y, mh.y);
                mh.z = fmaf(w, m.z, mh.z);
                mh.w = fmaf(w, m.w, mh.w);
                hmin = min(hmin, hv[t]);
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
        S::put_mom(mom_out, p, m, s);
        hist_out[p] = (uint8_t)n;
        if (n >= 4)
            illum[p] = make_float4(c.x, c.y, fmaxf(0.f, m.z - m.x * m.x), fmaxf(0.f, m.w - m.y * m.y));
    } else if (inside) {
        illum[p] = make_float4(1.f, 1.f, -1.f, -1.f);
        S::put_mom(mom_out, p, make_float4(1.f, 1.f, 1.f, 1.f), make_float2(1.f, 1.f));
        hist_out[p] = 0;
    }
    // short history (n < 4): 7x7 spatial estimate of the current frame's
    // signal weighted by depth and normal only.  With few such lanes in the
    // warp they are served one after another by the whole warp (lane l takes
    // taps l and l + 32 of the 49, then the sums are reduced across the
    // warp); with many, each lane sums its own 49 taps.
    const bool need = fg && n < 4;
    unsigned todo = __ballot_sync(kFull, need);
    if (__popc(todo) >= kShortPerLane) {
        // many short-history lanes (first frames, large disocclusions): each
        // computes its own 49 taps, cheaper than one warp pass per lane
        if (need) {
            float sw = 0.f, a1 = 0.f, b1 = 0.f, a2 = 0.f, b2 = 0.f;
            const float3 np = make_float3(zn.y, zn.z, zn.w);
            for (int dy = -3; dy <= 3; ++dy) {
                const int qy = y + dy;
                if (qy < 0 || qy >= k.H) continue;
#pragma unroll
                for (int dx = -3; dx <= 3; ++dx) {
                    const int qx = x + dx;
                    if (qx < 0 || qx >= k.W) continue;
                    const int q = (int)dbg_index((long long)qy * k.W + qx, (long long)k.W * k.H, kSiteShortHist);
                    const float4 zq = S::g(g_cur, q);
                    const float2 sq = sig(q);
                    if (!is_fg(zq.x)) continue;
                    const float w = w_spatial(k, zn.x, np, gz, dx, dy, zq);
                    sw += w;
                    a1 = fmaf(w, sq.x, a1);
                    b1 = fmaf(w, sq.y, b1);
                    a2 = fmaf(w, sq.x * sq.x, a2);
                    b2 = fmaf(w, sq.y * sq.y, b2);
                }
            }
            const float m1x = a1 / sw, m1y = b1 / sw;
            illum[p] = make_float4(m1x, m1y, fmaxf(0.f, a2 / sw - m1x * m1x), fmaxf(0.f, b2 / sw - m1y * m1y));
        }
        return;
    }
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int px = __shfl_sync(kFull, x, src), py = __shfl_sync(kFull, y, src);
        const float zp = __shfl_sync(kFull, zn.x, src);
        const float nx = __shfl_sync(kFull, zn.y, src), ny = __shfl_sync(kFull, zn.z, src),
                    nz = __shfl_sync(kFull, zn.w, src);
        const float gx = __shfl_sync(kFull, gz.x, src), gy = __shfl_sync(kFull, gz.y, src);
        float sw = 0.f, a1 = 0.f, b1 = 0.f, a2 = 0.f, b2 = 0.f;
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const int t = lane + 32 * it;
            const int dx = t % 7 - 3, dy = t / 7 - 3;
            const int qx = px + dx, qy = py + dy;
            if (t >= 49 || qx < 0 || qy < 0 || qx >= k.W || qy >= k.H) continue;
            const int q = (int)dbg_index((long long)qy * k.W + qx, (long long)k.W * k.H, kSiteShortHist);
            const float4 zq = S::g(g_cur, q);
            const float2 sq = sig(q);
            if (!is_fg(zq.x)) continue;
            const float w = w_spatial(k, zp, make_float3(nx, ny, nz), make_float2(gx, gy), dx, dy, zq);
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
__global__ void __launch_bounds__(256, 5) temporal_kernel(
    SvgfConsts k, dhr_camera cam, dhr_camera cam_prev, const typename Store<P>::G* g_cur,
    const uint32_t* mesh_cur, const typename Store<P>::G* g_prev, const uint32_t* mesh_prev,
    Sig sig, const typename Store<P>::Col* col_hist,
    const typename Store<P>::Mom* mom_in, const uint8_t* hist_in, typename Store<P>::Mom* mom_out,
    uint8_t* hist_out, float4* illum) {
    temporal_tile<P, Sig>(k, cam, cam_prev, g_cur, mesh_cur, g_prev, mesh_prev, sig, col_hist, mom_in, hist_in,
                          mom_out, hist_out, illum, blockIdx.x * 32, blockIdx.y * 8);
}

// log2 of the normal weight max(0, c)^sigma_n: -inf when c <= 0 (weight 0),
// 0 when sigma_n == 0 (weight 1, the 0^0 = 1 convention)
template <int kNsq>
__device__ __forceinline__ float log2_normal(float c, float sigma_n) {
    const float l = lg2_approx(fmaxf(c, 0.0f));
    if constexpr (kNsq >= 0) return (float)(1 << kNsq) * l;
    else return sigma_n == 0.0f ? 0.0f : sigma_n * l;
}

// Tiling of one a-trous iteration at step s.
//
// Step 1: a block takes a 32x8 pixel tile and stages the 36x12 pixels
// around it (illum and G-buffer) in shared memory once; the 24 taps, the
// 3x3 variance Gaussian and the depth gradient of every pixel then read
// shared memory only.  Pixels outside the image are staged as background
// (variance -1, depth +inf), which gives them weight exactly 0, as if they
// were skipped.
//
// Steps >= 2: the 5x5 footprint spans 4s + 1 pixels, so a staged tile
// would mostly hold halo; the taps are loaded directly (L1/L2 hits: the
// level's input and G-buffer stay resident in L2) and the per-pixel terms
// come from the pixel's immediate neighbours, which adjacent threads share.
//
// Both cover the image with the same 32x8 tiles, ceil(W/32) x ceil(H/8).
constexpr int kAtW = 32, kAtH = 8, kAtHalo = 2;
constexpr int kAtSW = kAtW + 2 * kAtHalo, kAtSH = kAtH + 2 * kAtHalo;

struct AtrousSmem {
    float4 c[kAtSH][kAtSW];    // (ao, shadow, var_ao, var_shadow)
    float4 g[kAtSH][kAtSW];    // (depth, normal)
};

__host__ __device__ inline int atrous_tiles_x(int W) { return (W + kAtW - 1) / kAtW; }
__host__ __device__ inline int atrous_tiles(int W, int H) { return atrous_tiles_x(W) * ((H + kAtH - 1) / kAtH); }

// per-axis depth slope (minmod of the one-sided differences) from the four
// neighbour depths (+inf: background or outside the image)
__device__ __forceinline__ float2 grad_from(float zp, float zxp, float zxm, float zyp, float zym) {
    const float n[2][2] = {{zxp, zxm}, {zyp, zym}};
    float r[2];
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
        const bool hp = is_fg(n[ax][0]), hm = is_fg(n[ax][1]);
        const float dp = hp ? n[ax][0] - zp : 0.f, dm = hm ? zp - n[ax][1] : 0.f;
        r[ax] = minmod_slope(hp, dp, hm, dm);
    }
    return make_float2(r[0], r[1]);
}

// tap sources: the staged tile, or the buffers (with or without bounds
// tests; a tap outside the image reads as background)
struct TapsSmem {
    const AtrousSmem& sm;
    int tx, ty;
    __device__ __forceinline__ void operator()(int i, int j, float4& c, float4& z) const {
        c = sm.c[ty + j][tx + i];
        z = sm.g[ty + j][tx + i];
    }
};

template <class S, bool kCheck>
struct TapsGlobal {
    const typename S::G* g;
    const float4* in;
    int W, H, x, y, step;
    __device__ __forceinline__ void operator()(int i, int j, float4& c, float4& z) const {
        const int qx = x + i * step, qy = y + j * step;
        if (kCheck && (qx < 0 || qy < 0 || qx >= W || qy >= H)) {
            c = make_float4(1.f, 1.f, -1.f, -1.f);
            z = make_float4(INFINITY, 0.f, 0.f, 0.f);
            return;
        }
        const int q = (int)dbg_index((long long)qy * W + qx, (long long)W * H, kSiteAtrousTap);
        c = __ldg(in + q);
        z = S::g(g, q);
    }
};

// The weighted sums of one pixel over its 5x5 footprint.  Each tap's weight
// for channel c, h_i h_j w_n w_z w_l,c, is evaluated as one power of two,
//   2^(log2(h_i h_j) + sigma_n log2(n.n_q) - |dz| rz - |dc| il_c)
// (rz and il_c carry log2(e)): one lg2 per tap and one ex2 per channel.
// Background taps (depth +inf, outside the image staged likewise) get
// |dz| rz = +inf, so exponent -inf and weight exactly 0; their illum holds
// the finite sentinel (1, 1, -1, -1), so the sums stay unchanged.
struct AtrousSums {
    float sw0, sw1, sc0, sc1, sv0, sv1;
};

// Footprint radius kR: 2 for the 5x5 B3-spline taps (1/16, 1/4, 3/8, 1/4,
// 1/16), 1 for the 3x3 taps (1/4, 1/2, 1/4) of the lightweight variant.
template <int kR>
struct AtrousTaps;
template <>
struct AtrousTaps<2> {
    // log2 of the taps; centre weight (3/8)^2
    static __device__ __forceinline__ float lg(int i) {
        return i == 0 ? -1.41503750f : ((i == 1 || i == -1) ? -2.f : -4.f);
    }
    static constexpr float kc = 0.375f * 0.375f;
};
template <>
struct AtrousTaps<1> {
    static __device__ __forceinline__ float lg(int i) { return i == 0 ? -1.f : -2.f; }
    static constexpr float kc = 0.25f;
};

template <int kNsq, int kR, class Taps>
__device__ __forceinline__ AtrousSums atrous_sums(const SvgfConsts& k, int step, float4 cp, float4 zn, float gv0,
                                                  float gv1, float gw, float2 gz, const Taps& taps) {
    constexpr int kD = 2 * kR + 1, kHalf = kD * kD / 2 + 1;
    // luminance terms folded with log2(e): w_l = 2^(-|dc| il)
    const float rgw = rcp_approx(gw);
    const float il0 = k.wl_in_atrous ? kLog2e * rcp_approx(fmaf(k.sigma_l, sqrt_approx(gv0 * rgw), k.eps_l)) : 0.f;
    const float il1 = k.wl_in_atrous ? kLog2e * rcp_approx(fmaf(k.sigma_l, sqrt_approx(gv1 * rgw), k.eps_l)) : 0.f;
    // depth terms: log2(e) / (sigma_z |grad z . (p - q)| + eps_z) for the
    // offset directions (i, j) ~ (-i, -j) of the footprint
    const float sg = k.sigma_z * (float)step;
    float rz[kHalf];
#pragma unroll
    for (int m = 0; m < kHalf; ++m) {
        const int i = m % kD - kR, j = m / kD - kR;    // j < 0, or j = 0 and i < 0 (+ the centre, last)
        rz[m] = kLog2e * rcp_approx(fmaf(sg, fabsf(fmaf(gz.x, (float)i, gz.y * (float)j)), k.eps_z));
    }
    constexpr float kc = AtrousTaps<kR>::kc;
    // the two channels' sums (w, w c, w^2 var) as f32x2 pairs
    unsigned long long sw = pack2(kc, kc), sc = pack2(kc * cp.x, kc * cp.y);
    unsigned long long sv = pack2(kc * kc * cp.z, kc * kc * cp.w);
#pragma unroll
    for (int j = -kR; j <= kR; ++j) {
#pragma unroll
        for (int i = -kR; i <= kR; ++i) {
            if (i == 0 && j == 0) continue;
            float4 cq, zq;
            taps(i, j, cq, zq);
            const int m = (j < 0 || (j == 0 && i < 0)) ? (j + kR) * kD + (i + kR) : (kR - j) * kD + (kR - i);
            float e = fmaf(-fabsf(zn.x - zq.x), rz[m], AtrousTaps<kR>::lg(i) + AtrousTaps<kR>::lg(j));
            e += log2_normal<kNsq>(zn.y * zq.y + zn.z * zq.z + zn.w * zq.w, k.sigma_n);
            const unsigned long long w = pack2(ex2_approx(fmaf(-fabsf(cp.x - cq.x), il0, e)),
                                               ex2_approx(fmaf(-fabsf(cp.y - cq.y), il1, e)));
            sw = add2(sw, w);
            sc = fma2(w, pack2(cq.x, cq.y), sc);
            sv = fma2(mul2(w, w), pack2(cq.z, cq.w), sv);
        }
    }
    const float2 w = unpack2(sw), c = unpack2(sc), v = unpack2(sv);
    return AtrousSums{w.x, w.y, c.x, c.y, v.x, v.y};
}

// 3x3 Gaussian of the variance, renormalised over foreground taps; v[dy][dx]
__device__ __forceinline__ void var_gauss(const float4 (&v)[3][3], float& gv0, float& gv1, float& gw) {
    gv0 = gv1 = gw = 0.f;
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
            if (!fg_var(v[dy][dx].z)) continue;
            const float kk = (dx == 1 ? 0.5f : 0.25f) * (dy == 1 ? 0.5f : 0.25f);
            gw += kk;
            gv0 = fmaf(kk, v[dy][dx].z, gv0);
            gv1 = fmaf(kk, v[dy][dx].w, gv1);
        }
}

// Records of one level for the differentiable form (both null outside it):
// the weight sums (sum w per channel, centre included) and, for the last
// level, its filtered colour and variance, which no later level keeps.
struct AtrousRec {
    float2* wsum;
    float4* last;
};

template <dhr_precision P, int kMode, bool kRec = false>
__device__ __forceinline__ void atrous_store(const AtrousSums& a, int p, float4* out,
                                             typename Store<P>::Col* col_hist, float* ao_out, float* sh_out,
                                             AtrousRec rec = AtrousRec{nullptr, nullptr}) {
    // (sum w c) / (sum w) correctly rounded: a constant neighbourhood stays
    // exactly constant; the variance (sum w^2 v) / (sum w)^2 needs no such care
    const float c0 = a.sc0 / a.sw0, c1 = a.sc1 / a.sw1;
    if (kRec) rec.wsum[p] = make_float2(a.sw0, a.sw1);
    if (kMode == 2) {
        if (!kRec || ao_out) {   // a recording pass may only want the records
            ao_out[p] = c0;
            sh_out[p] = c1;
        }
        if (kRec) {
            const float r0 = rcp_approx(a.sw0), r1 = rcp_approx(a.sw1);
            rec.last[p] = make_float4(c0, c1, a.sv0 * r0 * r0, a.sv1 * r1 * r1);
        }
    } else {
        const float r0 = rcp_approx(a.sw0), r1 = rcp_approx(a.sw1);
        out[p] = make_float4(c0, c1, a.sv0 * r0 * r0, a.sv1 * r1 * r1);
        if (kMode == 1) Store<P>::put_col(col_hist, p, make_float2(c0, c1));
    }
}

template <dhr_precision P, int kMode, bool kRec = false>
__device__ __forceinline__ void atrous_background(int p, float4* out, typename Store<P>::Col* col_hist,
                                                  float* ao_out, float* sh_out) {
    if (kMode == 2) {
        if (!kRec || ao_out) {
            ao_out[p] = 1.f;
            sh_out[p] = 1.f;
        }
    } else {
        out[p] = make_float4(1.f, 1.f, -1.f, -1.f);
        if (kMode == 1) Store<P>::put_col(col_hist, p, make_float2(1.f, 1.f));
    }
}

// One a-trous iteration over the 32x8 tile t; kMode 0: write illum_out;
// 1: also the colour history; 2: last iteration, write the two output
// planes only.  kNsq >= 0: sigma_n is 2^kNsq.  kR: footprint radius (2:
// 5x5, 1: 3x3).  Every thread of the block must call it (block barriers at
// step 1).
template <dhr_precision P, int kMode, int kNsq, int kR = 2, bool kRec = false>
__device__ __forceinline__ void atrous_tile(const SvgfConsts& k, int step, int t, const typename Store<P>::G* g,
                                            const float4* in, float4* out, typename Store<P>::Col* col_hist,
                                            float* ao_out, float* sh_out, AtrousSmem& sm,
                                            AtrousRec rec = AtrousRec{nullptr, nullptr}) {
    using S = Store<P>;
    const int ntx = atrous_tiles_x(k.W);
    const int bx0 = (t % ntx) * kAtW, by0 = (t / ntx) * kAtH;
    const int x = bx0 + (int)threadIdx.x, y = by0 + (int)threadIdx.y;
    const bool inside = x < k.W && y < k.H;
    const int p = y * k.W + x;
    if (step == 1) {
        for (int i = threadIdx.y * kAtW + threadIdx.x; i < kAtSW * kAtSH; i += kAtW * kAtH) {
            const int sy = i / kAtSW, sx = i - sy * kAtSW;
            const int qx = bx0 - kAtHalo + sx, qy = by0 - kAtHalo + sy;
            float4 c = make_float4(1.f, 1.f, -1.f, -1.f), z = make_float4(INFINITY, 0.f, 0.f, 0.f);
            if (qx >= 0 && qy >= 0 && qx < k.W && qy < k.H) {
                const int q = (int)dbg_index((long long)qy * k.W + qx, (long long)k.W * k.H, kSiteAtrousTap);
                c = __ldg(in + q);
                z = S::g(g, q);
            }
            sm.c[sy][sx] = c;
            sm.g[sy][sx] = z;
        }
        __syncthreads();
        const int tx = threadIdx.x + kAtHalo, ty = threadIdx.y + kAtHalo;
        const float4 cp = sm.c[ty][tx];
        if (inside) {
            if (!fg_var(cp.z)) {
                atrous_background<P, kMode, kRec>(p, out, col_hist, ao_out, sh_out);
            } else {
                const float4 zn = sm.g[ty][tx];
                float4 v[3][3];
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) v[dy][dx] = sm.c[ty + dy - 1][tx + dx - 1];
                float gv0, gv1, gw;
                var_gauss(v, gv0, gv1, gw);
                const float2 gz = grad_from(zn.x, sm.g[ty][tx + 1].x, sm.g[ty][tx - 1].x, sm.g[ty + 1][tx].x,
                                            sm.g[ty - 1][tx].x);
                const AtrousSums a = atrous_sums<kNsq, kR>(k, 1, cp, zn, gv0, gv1, gw, gz, TapsSmem{sm, tx, ty});
                atrous_store<P, kMode, kRec>(a, p, out, col_hist, ao_out, sh_out, rec);
            }
        }
        __syncthreads();    // the staging area is reused by the block's next tile
        return;
    }
    if (!inside) return;
    const float4 cp = __ldg(in + p);
    if (!fg_var(cp.z)) {
        atrous_background<P, kMode, kRec>(p, out, col_hist, ao_out, sh_out);
        return;
    }
    const float4 zn = S::g(g, p);
    float4 v[3][3];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int qx = x + dx, qy = y + dy;
            v[dy + 1][dx + 1] =
                (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H)
                    ? make_float4(1.f, 1.f, -1.f, -1.f)
                    : __ldg(in + dbg_index((long long)qy * k.W + qx, (long long)k.W * k.H, kSiteAtrousVar));
        }
    float gv0, gv1, gw;
    var_gauss(v, gv0, gv1, gw);
    const float2 gz = grad_from(zn.x, x + 1 < k.W ? S::g(g, p + 1).x : INFINITY, x > 0 ? S::g(g, p - 1).x : INFINITY,
                                y + 1 < k.H ? S::g(g, p + k.W).x : INFINITY, y > 0 ? S::g(g, p - k.W).x : INFINITY);
    // blocks whose footprint lies inside the image skip the bounds tests
    const int reach = kR * step;
    const bool interior = bx0 - reach >= 0 && by0 - reach >= 0 && bx0 + kAtW - 1 + reach < k.W &&
                          by0 + kAtH - 1 + reach < k.H;
    AtrousSums a;
    if (interior)
        a = atrous_sums<kNsq, kR>(k, step, cp, zn, gv0, gv1, gw, gz,
                                  TapsGlobal<S, false>{g, in, k.W, k.H, x, y, step});
    else
        a = atrous_sums<kNsq, kR>(k, step, cp, zn, gv0, gv1, gw, gz,
                                  TapsGlobal<S, true>{g, in, k.W, k.H, x, y, step});
    atrous_store<P, kMode, kRec>(a, p, out, col_hist, ao_out, sh_out, rec);
}

template <dhr_precision P, int kMode, int kNsq, int kR, bool kRec = false>
__global__ void __launch_bounds__(256, 4) atrous_kernel(SvgfConsts k, int step, const typename Store<P>::G* g,
                                                     const float4* in, float4* out,
                                                     typename Store<P>::Col* col_hist, float* ao_out,
                                                     float* sh_out, AtrousRec rec) {
    __shared__ AtrousSmem sm;
    atrous_tile<P, kMode, kNsq, kR, kRec>(k, step, blockIdx.x, g, in, out, col_hist, ao_out, sh_out, sm, rec);
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
    k.shadow_bit = prm->shadow_light;
    return k;
}

inline int atrous_nsq(const dhr_svgf_params* prm) { return prm->sigma_n == 128.0f ? 7 : -1; }

// footprint radius of the a-trous taps: 1 for kernel_width 3, else 2 (5x5)
inline int atrous_radius(const dhr_svgf_params* prm) { return prm->kernel_width == 3 ? 1 : 2; }

template <dhr_precision P, int kMode, int kR>
inline void launch_atrous_mode(int nsq, cudaStream_t st, const SvgfConsts& k, int step,
                               const typename Store<P>::G* g, const float4* in, float4* out,
                               typename Store<P>::Col* col, float* ao_out, float* sh_out) {
    const dim3 grid(atrous_tiles(k.W, k.H)), blk(kAtW, kAtH);
    const AtrousRec none{nullptr, nullptr};
    if (nsq == 7)
        atrous_kernel<P, kMode, 7, kR><<<grid, blk, 0, st>>>(k, step, g, in, out, col, ao_out, sh_out, none);
    else
        atrous_kernel<P, kMode, -1, kR><<<grid, blk, 0, st>>>(k, step, g, in, out, col, ao_out, sh_out, none);
}

template <dhr_precision P, int kR>
inline void launch_atrous_r(int mode, int nsq, cudaStream_t st, const SvgfConsts& k, int step,
                            const typename Store<P>::G* g, const float4* in, float4* out,
                            typename Store<P>::Col* col, float* ao_out, float* sh_out) {
    if (mode == 2)
        launch_atrous_mode<P, 2, kR>(nsq, st, k, step, g, in, nullptr, nullptr, ao_out, sh_out);
    else if (mode == 1)
        launch_atrous_mode<P, 1, kR>(nsq, st, k, step, g, in, out, col, nullptr, nullptr);
    else
        launch_atrous_mode<P, 0, kR>(nsq, st, k, step, g, in, out, nullptr, nullptr, nullptr);
}

// one a-trous iteration at `step` over the whole W x H image of `k`, with
// footprint radius R (2: 5x5, 1: 3x3)
template <dhr_precision P>
inline dhr_status launch_atrous(int mode, int nsq, int R, cudaStream_t st, const SvgfConsts& k, int step,
                                const typename Store<P>::G* g, const float4* in, float4* out,
                                typename Store<P>::Col* col, float* ao_out, float* sh_out) {
    if (R == 1)
        launch_atrous_r<P, 1>(mode, nsq, st, k, step, g, in, out, col, ao_out, sh_out);
    else
        launch_atrous_r<P, 2>(mode, nsq, st, k, step, g, in, out, col, ao_out, sh_out);
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}

// The differentiable form's forward level (binary32, 5x5): as launch_atrous,
// plus the level's records `rec` (wsum always; last on mode 2).  Mode 2
// with null ao_out / sh_out writes the records only.
inline dhr_status launch_atrous_recorded(int mode, int nsq, cudaStream_t st, const SvgfConsts& k, int step,
                                         const float4* g, const float4* in, float4* out, float2* col, float* ao_out,
                                         float* sh_out, AtrousRec rec) {
    const dim3 grid(atrous_tiles(k.W, k.H)), blk(kAtW, kAtH);
    constexpr dhr_precision P = DHR_FP32;
#define DHR_ATROUS_REC(M, NSQ, OUT, COL, AO, SH) \
    atrous_kernel<P, M, NSQ, 2, true><<<grid, blk, 0, st>>>(k, step, g, in, OUT, COL, AO, SH, rec)
    if (mode == 2) {
        if (nsq == 7) DHR_ATROUS_REC(2, 7, nullptr, nullptr, ao_out, sh_out);
        else DHR_ATROUS_REC(2, -1, nullptr, nullptr, ao_out, sh_out);
    } else if (mode == 1) {
        if (nsq == 7) DHR_ATROUS_REC(1, 7, out, col, nullptr, nullptr);
        else DHR_ATROUS_REC(1, -1, out, col, nullptr, nullptr);
    } else {
        if (nsq == 7) DHR_ATROUS_REC(0, 7, out, nullptr, nullptr, nullptr);
        else DHR_ATROUS_REC(0, -1, out, nullptr, nullptr, nullptr);
    }
#undef DHR_ATROUS_REC
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}

}  // namespace dhr
