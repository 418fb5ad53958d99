// Adjoint of the modified SVGF (Section 3.3) over a sequence of frames.
//
// The paper has no gradient; this is the differentiable form of its filter:
// a loss on the filtered colour is back-propagated to the per-pixel noisy
// signals (AO, shadow) of every frame and to the edge-stopping parameters
// sigma_z, sigma_n, sigma_l, through all a-trous levels, the variance
// estimate, the moving averages and the reprojected history of earlier
// frames (the temporal recursion is not cut).
//
// Forward (dhr_svgf_seq_forward) records per frame the temporal output
// (colour, variance), the moments and the history lengths.  The level
// records a frame's adjoint reads -- the input of every a-trous level after
// the first, every level's weight sums and the last level's output -- are
// recomputed from the temporal output by the backward, one frame ahead on a
// low-priority stream while the passes run on a high-priority one (the
// forward leaves the last two frames' in place), or kept for every frame by
// the forward (DHR_TAPE_STORE).  Backward of one a-trous
// level is a two-pass gather:
//   pass A (per output pixel p): with the level's weight sum, filtered
//     colour and variance at p from the forward, dL/dw_pq = a1 c_q - a2 +
//     a3 w_pq v_q is known tap by tap, so one pass over p's taps forms the
//     gradient through p's own colour and p's luminance scale and the sigma
//     derivatives;
//   pass B (per input pixel q): gather from the 24 pixels whose footprint
//     contains q (weights rebuilt from the G-buffer and the records) and
//     from the 9 whose variance Gaussian does.
// The reprojection taps and history lengths depend only on G-buffers and
// cameras and are constants of the adjoint.  Conventions as in the CPU
// reference: sign(0) = 0, d max(0, x) = [x > 0], d sqrt(g)/dg = 0 for g < 1e-12,
// d w_n/d sigma_n = w_n ln(n.n') for n.n' > 0.
#include <vector>

#include "svgf_kernels.cuh"

namespace dhr {
namespace {

constexpr int kBX = 32, kBY = 8, kThreadsA = kBX * kBY;

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

constexpr float kLn2 = 0.69314718055994531f;

using u64 = unsigned long long;

// records of pass A, four planes of one float4 per pixel (rec[r * N + p],
// so that a warp's loads of one plane are contiguous), channel pairs adjacent:
//   r0 = (a1[0], a1[1], -a2[0], -a2[1]), r1 = (a3[0], a3[1], il[0], il[1]),
//   r2 = (Gg[0], Gg[1], self[0], self[1]), r3 = (grad z, c[0], c[1])
// (Gg already divided by the pixel's Gaussian normaliser; zero records on
// background pixels, whose infinite depth gives every tap of theirs weight
// 0 in pass B).  gs[p] += this level's (dL/d sigma_z, dL/d sigma_n,
// dL/d sigma_l) terms of pixel p.
//
// dL/dw_pq = a1 c_q - a2 + a3 w_pq v_q with a1 = G_c / W, a2 = (G_c c +
// 2 G_v v) / W, a3 = 2 G_v / W^2, where W, c and v are the level's weight
// sum, filtered colour and filtered variance at p (the forward's records),
// so one pass over the taps forms every derivative.  Both channels at once
// as packed binary32 pairs (lane 0: AO, lane 1: shadow; each lane rounded
// as the scalar operation).
// The colour-free part of log2 w_pq for tap (i, j) of p (q = p + (i, j) step):
//   log2(h_i h_j) + sigma_n log2(n_p . n_q) - log2(e) |z_p - z_q| / D,
// D = sigma_z step |grad z_p . (i, j)| + eps_z; with the factors the sigma
// derivatives reuse (u = |z_p - z_q| / D, a_off, rD = 1 / D, nd, log2 nd).
struct TapLog {
    float e, u, a_off, rD, nd, l2n;
};

template <int kNsq>
__device__ __forceinline__ TapLog tap_log(const SvgfConsts& k, int step, int i, int j, float4 zp, float2 gz,
                                          float4 zq) {
    const float l5[5] = {-4.f, -2.f, -1.41503750f, -2.f, -4.f};
    TapLog t;
    t.a_off = (float)step * fabsf(fmaf(gz.x, (float)i, gz.y * (float)j));
    t.rD = rcp_approx(fmaf(k.sigma_z, t.a_off, k.eps_z));
    t.u = fabsf(zp.x - zq.x) * t.rD;
    t.nd = zp.y * zq.y + zp.z * zq.z + zp.w * zq.w;
    t.l2n = lg2_approx(fmaxf(t.nd, 0.0f));
    float en;
    if constexpr (kNsq >= 0) en = (float)(1 << kNsq) * t.l2n;
    else en = k.sigma_n == 0.0f ? 0.0f : k.sigma_n * t.l2n;
    t.e = fmaf(-kLog2e, t.u, l5[i + 2] + l5[j + 2]) + en;
    return t;
}

template <int kNsq, bool kLum, bool kCheck>
__device__ __forceinline__ void bwd_a_pixel(const SvgfConsts& k, int step, const float4* g, const float4* x,
                                            float2 Gc, float2 Gv, float2 W, float4 out, float4* rec, float4* gs,
                                            size_t N, int px, int py, int p, float4 cp) {
    using S = Store<DHR_FP32>;
    const float4 zp = S::g(g, p);
    float gv0 = 0.f, gv1 = 0.f, gw = 0.f;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int qx = px + dx, qy = py + dy;
            if (kCheck && (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H)) continue;
            const float4 v = __ldg(x + dbg_index((long long)qy * k.W + qx, (long long)N, kSiteAdjoint));
            if (!fg_var(v.z)) continue;
            const float kk = (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f);
            gw += kk;
            gv0 = fmaf(kk, v.z, gv0);
            gv1 = fmaf(kk, v.w, gv1);
        }
    const float root0 = sqrtf(fmaxf(0.f, gv0 / gw)), root1 = sqrtf(fmaxf(0.f, gv1 / gw));
    const float il0 = kLum ? 1.0f / (k.sigma_l * root0 + k.eps_l) : 0.f;
    const float il1 = kLum ? 1.0f / (k.sigma_l * root1 + k.eps_l) : 0.f;
    const float nil0 = -kLog2e * il0, nil1 = -kLog2e * il1;
    const float2 gz = depth_grad<S>(g, k.W, k.H, px, py, zp.x);
    const float rW0 = 1.0f / W.x, rW1 = 1.0f / W.y;
    const float a10 = Gc.x * rW0, a11 = Gc.y * rW1;
    const float a20 = (Gc.x * out.x + 2.f * Gv.x * out.z) * rW0, a21 = (Gc.y * out.y + 2.f * Gv.y * out.w) * rW1;
    const float a30 = 2.f * Gv.x * rW0 * rW0, a31 = 2.f * Gv.y * rW1 * rW1;
    const u64 A1 = pack2(a10, a11), NA2 = pack2(-a20, -a21), A3 = pack2(a30, a31);
    u64 self_s = 0, gil_s = 0;   // sum dL/dw w sgn(c_q - c_p), sum dL/dw w |c_q - c_p|
    float gsz = 0.f, gsn = 0.f;
#pragma unroll
    for (int j = -2; j <= 2; ++j)
#pragma unroll
        for (int i = -2; i <= 2; ++i) {
            if (!i && !j) continue;
            const int qx = px + i * step, qy = py + j * step;
            if (kCheck && (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H)) continue;
            const int q = (int)dbg_index((long long)qy * k.W + qx, (long long)N, kSiteAdjoint);
            const float4 cq = __ldg(x + q);
            // interior tiles issue both loads before testing the tap: a
            // background tap (depth +inf, finite colour sentinel) gets weight
            // exactly 0, and its sigma_z term is selected away
            const float4 zq = S::g(g, q);
            const bool fg = fg_var(cq.z);
            if (kCheck && !fg) continue;
            const TapLog t = tap_log<kNsq>(k, step, i, j, zp, gz, zq);
            const float d0 = cq.x - cp.x, d1 = cq.y - cp.y;
            const u64 w = pack2(ex2_approx(fmaf(nil0, fabsf(d0), t.e)), ex2_approx(fmaf(nil1, fabsf(d1), t.e)));
            const u64 Gw = fma2(mul2(A3, w), pack2(cq.z, cq.w), fma2(A1, pack2(cq.x, cq.y), NA2));
            const u64 gww = mul2(Gw, w);
            if (kLum) {
                self_s = fma2(gww, pack2(sgnf(d0), sgnf(d1)), self_s);
                gil_s = fma2(gww, pack2(fabsf(d0), fabsf(d1)), gil_s);
            }
            const float2 gf = unpack2(gww);
            const float gsum = gf.x + gf.y;
            // d w / d sigma_z = w |dz| a_off / D^2;  d w / d sigma_n = w ln(n . n_q)
            gsz = fmaf(gsum, fg ? t.u * t.a_off * t.rD : 0.f, gsz);
            if (t.nd > 0.f) gsn = fmaf(gsum, t.l2n, gsn);
        }
    float4 acc = gs[p];
    acc.x += gsz;
    acc.y += gsn * kLn2;
    float Gg0 = 0.f, Gg1 = 0.f, self0 = 0.f, self1 = 0.f;
    if (kLum) {
        const float2 ss = unpack2(self_s), ga = unpack2(gil_s);
        // d w / d c_p = -w il sgn(c_p - c_q) = w il sgn(c_q - c_p)
        self0 = il0 * ss.x;
        self1 = il1 * ss.y;
        // d w / d il = -w |c_p - c_q|
        const float Gil0 = -ga.x, Gil1 = -ga.y;
        acc.z += Gil0 * (-il0 * il0 * root0) + Gil1 * (-il1 * il1 * root1);
        // d sqrt(g)/dg is taken as 0 below g = 1e-12 (it grows without bound
        // toward g = 0, where the weight is already insensitive)
        if (root0 > 1e-6f) Gg0 = Gil0 * (-il0 * il0 * k.sigma_l * 0.5f / root0) / gw;
        if (root1 > 1e-6f) Gg1 = Gil1 * (-il1 * il1 * k.sigma_l * 0.5f / root1) / gw;
    }
    gs[p] = acc;
    rec[p] = make_float4(a10, a11, -a20, -a21);
    rec[N + p] = make_float4(a30, a31, il0, il1);
    rec[2 * N + p] = make_float4(Gg0, Gg1, self0, self1);
    rec[3 * N + p] = make_float4(gz.x, gz.y, cp.x, cp.y);
}

// 32x8 pixel tiles; a tile whose taps (reach 2 step) and 3x3 variance
// neighbourhoods all lie inside the image skips the bounds tests
__device__ __forceinline__ bool tile_interior(const SvgfConsts& k, int step, int bx, int by) {
    const int reach = 2 * step, bx0 = bx * kBX, by0 = by * kBY;
    return bx0 - reach >= 0 && by0 - reach >= 0 && bx0 + kBX - 1 + reach < k.W && by0 + kBY - 1 + reach < k.H;
}

// pass B: gradient with respect to the level's input colour and variance.
// The taps are evaluated without branches (a tap outside the image reads the
// centre's own records, and a select drops it; a background tap has zero
// records and weight 0) so that the loads of all taps can be issued
// together.  The colour-free log-weight of each tap is recomputed from the
// G-buffer and the tapping pixel's recorded depth gradient.
// Returns (dL/d c_q, dL/d v_q) per channel.
template <int kNsq, bool kCheck>
__device__ __forceinline__ float4 bwd_b_pixel(const SvgfConsts& k, int step, const float4* g, const float4* rec,
                                              size_t N, int qx, int qy, int q, float4 cq) {
    using S = Store<DHR_FP32>;
    const float kc = 0.375f * 0.375f;
    const float4 r0 = rec[q], r1 = rec[N + q], r2 = rec[2 * N + q];
    // own colour through the weights of q's own footprint, and the centre tap
    u64 gcs = pack2(r2.z + r0.x * kc, r2.w + r0.y * kc);
    u64 gvs = pack2(0.5f * r1.x * kc * kc, 0.5f * r1.y * kc * kc);
    // variance Gaussians that read q (background pixels hold zero records)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int px = qx + dx, py = qy + dy;
            if (kCheck && (px < 0 || py < 0 || px >= k.W || py >= k.H)) continue;
            const float kk = (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f);
            const float4 rp = rec[2 * N + dbg_index((long long)py * k.W + px, (long long)N, kSiteAdjoint)];
            gvs = fma2(pack2(rp.x, rp.y), pack2(kk, kk), gvs);
        }
    const float4 zq = S::g(g, q);
    const u64 cqc = pack2(cq.x, cq.y), cqv = pack2(cq.z, cq.w), half = pack2(0.5f, 0.5f);
    const u64 ncq = pack2(-cq.x, -cq.y);
    // footprints of the 24 pixels p = q - (i, j) step that tap q at (i, j)
#pragma unroll
    for (int j = -2; j <= 2; ++j)
#pragma unroll
        for (int i = -2; i <= 2; ++i) {
            if (!i && !j) continue;
            const int px = qx - i * step, py = qy - j * step;
            const bool in = !kCheck || (px >= 0 && py >= 0 && px < k.W && py < k.H);
            const int p = (int)dbg_index(in ? (long long)py * k.W + px : q, (long long)N, kSiteAdjoint);
            const float4 p0 = rec[p], p1 = rec[N + p], p3 = rec[3 * N + p];
            const TapLog t = tap_log<kNsq>(k, step, i, j, S::g(g, p), make_float2(p3.x, p3.y), zq);
            const float2 d = unpack2(add2(pack2(p3.z, p3.w), ncq));   // c_p - c_q
            const float w0 = ex2_approx(fmaf(-kLog2e * p1.z, fabsf(d.x), t.e));
            const float w1 = ex2_approx(fmaf(-kLog2e * p1.w, fabsf(d.y), t.e));
            const u64 w = pack2(w0, w1);
            const u64 a3w = mul2(pack2(p1.x, p1.y), w);
            // dL/dw_pq = a1 c_q - a2 + a3 w v_q
            const u64 Gw = fma2(a3w, cqv, fma2(pack2(p0.x, p0.y), cqc, pack2(p0.z, p0.w)));
            const u64 sil = pack2(p1.z * sgnf(d.x), p1.w * sgnf(d.y));
            const float2 dc = unpack2(fma2(mul2(Gw, w), sil, mul2(pack2(p0.x, p0.y), w)));
            const float2 dv = unpack2(mul2(mul2(a3w, w), half));
            gcs = add2(gcs, pack2(in ? dc.x : 0.f, in ? dc.y : 0.f));
            gvs = add2(gvs, pack2(in ? dv.x : 0.f, in ? dv.y : 0.f));
        }
    const float2 gc = unpack2(gcs), gv = unpack2(gvs);
    return make_float4(gc.x, gc.y, gv.x, gv.y);
}

// Upstream gradient (dL/d colour, dL/d variance) of pixel q at the output
// of a level (or at the temporal output): from the loss gradient planes
// g_out [2][N] (the last level; no variance gradient) or from the buffers
// gc, gv that pass B of the level above wrote.  gcol (or null) adds the
// gradient that reaches level 0's output through the colour history of the
// next frame.
struct Upstream {
    const float* g_out;
    const float2* gc;
    const float2* gv;
    const float2* gcol;
};

__device__ __forceinline__ float4 upstream(const Upstream& up, size_t N, int q) {
    float4 G;
    if (up.g_out) {
        G = make_float4(up.g_out[q], up.g_out[N + q], 0.f, 0.f);
    } else {
        const float2 c = up.gc[q], v = up.gv[q];
        G = make_float4(c.x, c.y, v.x, v.y);
    }
    if (up.gcol) {
        const float2 a = up.gcol[q];
        G.x += a.x;
        G.y += a.y;
    }
    return G;
}

// wsum: the level's weight sums [N]; xout: its filtered colour and variance [N]
template <int kNsq, bool kLum>
__global__ void __launch_bounds__(kThreadsA, 4) atrous_bwd_a(SvgfConsts k, int step, const float4* g, const float4* x,
                                                             const float2* wsum, const float4* xout, Upstream up,
                                                             float4* rec, float4* gs) {
    const int px = blockIdx.x * kBX + threadIdx.x, py = blockIdx.y * kBY + threadIdx.y;
    if (px >= k.W || py >= k.H) return;
    const int p = py * k.W + px;
    const size_t N = (size_t)k.W * k.H;
    const float4 cp = __ldg(x + p);
    if (!fg_var(cp.z)) {
        rec[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec[N + p] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec[2 * N + p] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec[3 * N + p] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const float4 G = upstream(up, N, p);
    const float2 W = wsum[p];
    const float4 o = __ldg(xout + p);
    if (tile_interior(k, step, blockIdx.x, blockIdx.y))
        bwd_a_pixel<kNsq, kLum, false>(k, step, g, x, make_float2(G.x, G.y), make_float2(G.z, G.w), W, o, rec, gs, N,
                                       px, py, p, cp);
    else
        bwd_a_pixel<kNsq, kLum, true>(k, step, g, x, make_float2(G.x, G.y), make_float2(G.z, G.w), W, o, rec, gs, N,
                                      px, py, p, cp);
}

// Pass B runs its tiles in the reverse of pass A's order: the records pass
// A wrote last are the ones still in L2 when pass B starts.
template <int kNsq>
__global__ void __launch_bounds__(kThreadsA, 5) atrous_bwd_b(SvgfConsts k, int step, const float4* g, const float4* x,
                                                          const float4* rec, float2* gc_in, float2* gv_in) {
    const int bx = gridDim.x - 1 - blockIdx.x, by = gridDim.y - 1 - blockIdx.y;
    const int qx = bx * kBX + threadIdx.x, qy = by * kBY + threadIdx.y;
    if (qx >= k.W || qy >= k.H) return;
    const int q = qy * k.W + qx;
    const float4 cq = __ldg(x + q);
    if (!fg_var(cq.z)) {
        gc_in[q] = make_float2(0.f, 0.f);
        gv_in[q] = make_float2(0.f, 0.f);
        return;
    }
    const size_t N = (size_t)k.W * k.H;
    const float4 G = tile_interior(k, step, bx, by) ? bwd_b_pixel<kNsq, false>(k, step, g, rec, N, qx, qy, q, cq)
                                                    : bwd_b_pixel<kNsq, true>(k, step, g, rec, N, qx, qy, q, cq);
    gc_in[q] = make_float2(G.x, G.y);
    gv_in[q] = make_float2(G.z, G.w);
}

// Backward of the temporal step of one frame (FP32 storage).
//
// dL/d sig lands on the pixel itself (moving averages) and, for pixels with
// fewer than 4 frames of history, on the 7x7 neighbourhood of the spatial
// moment estimate.  The block accumulates both in a shared tile of its
// 32x8 pixels plus a 3-pixel apron and adds the tile to g_sig once, so the
// atomics to device memory are one per nonzero tile entry.  The history
// gradients scatter to the 4 reprojection taps of the previous frame with
// vector atomics (one float2 and one float4 per tap).
constexpr int kTR = 3, kTW = kBX + 2 * kTR, kTH = kBY + 2 * kTR;

// Weight of the 7x7 short-history estimate (the forward's w_spatial) with
// the intermediates its derivatives reuse: w = 2^(sigma_n log2(n.n_q) -
// log2(e) |dz| rD), rD = 1 / (sigma_z a_off + eps_z); the centre has w = 1.
struct W7 {
    float w, dz, a_off, rD, nd, l2n;
};

__device__ __forceinline__ W7 w7(const SvgfConsts& k, float4 zn, float2 gz, int dx, int dy, float4 zq) {
    W7 t;
    if (!(dx || dy)) {
        t.w = 1.0f;
        t.dz = t.a_off = t.l2n = 0.f;
        t.rD = t.nd = 1.f;
        return t;
    }
    t.a_off = fabsf(fmaf(gz.x, (float)-dx, gz.y * (float)-dy));
    t.rD = rcp_approx(fmaf(k.sigma_z, t.a_off, k.eps_z));
    t.dz = fabsf(zn.x - zq.x);
    t.nd = zn.y * zq.y + zn.z * zq.z + zn.w * zq.w;
    t.l2n = lg2_approx(fmaxf(t.nd, 0.0f));
    t.w = ex2_approx(fmaf(-t.dz, kLog2e * t.rD, k.sigma_n == 0.0f ? 0.0f : k.sigma_n * t.l2n));
    return t;
}

// Sums of the 7x7 estimate of one pixel: the weighted sums of w, s and s^2
// per channel (the forward's means).
struct Short7 {
    float sw, s1x, s1y, s2x, s2y;
};

// Adds tap (dx, dy) of pixel (x, y), read from the buffers (the warp-
// cooperative path).  The tap's loads are issued before it is tested: a tap
// outside the image reads the clamped pixel and is masked; a background tap
// (depth +inf) has weight exactly 0 and is masked likewise.
__device__ __forceinline__ void short7_tap(const SvgfConsts& k, const float4* g_cur, const float* sig, int N,
                                           float4 zn, float2 gz, int x, int y, int dx, int dy, Short7& a) {
    using S = Store<DHR_FP32>;
    const int qx = x + dx, qy = y + dy;
    const bool in = qx >= 0 && qy >= 0 && qx < k.W && qy < k.H;
    const long long qi = (long long)min(max(qy, 0), k.H - 1) * k.W + min(max(qx, 0), k.W - 1);
    const int q = (int)dbg_index(qi, (long long)N, kSiteAdjoint);
    const float4 zq = S::g(g_cur, q);
    const float sx = sig[q], sy = sig[N + q];
    const bool use = in && is_fg(zq.x);
    const float w = use ? w7(k, zn, gz, dx, dy, zq).w : 0.f;
    a.sw += w;
    a.s1x = fmaf(w, sx, a.s1x);
    a.s1y = fmaf(w, sy, a.s1y);
    a.s2x = fmaf(w, sx * sx, a.s2x);
    a.s2y = fmaf(w, sy * sy, a.s2y);
}

// Coefficients of the gradient with respect to tap q's signal and weight,
// from the sums and the gradient (Gc, Gv) at the estimate's colour and
// variance (colour = m1, var = max(0, m2 - m1^2), m_k = sum w s^k / sum w):
//   dL/d s_q = (G1 + 2 G2 s_q) w_q / sw per channel,
//   dL/d w_q = (G1 (s_q - m1) + G2 (s_q^2 - m2)) / sw summed over channels
//            = (c0 + sum_ch s_q (G1 + G2 s_q)) / sw.
struct ShortG {
    float G1x, G1y, G2x, G2y, c0, isw;
};

__device__ __forceinline__ ShortG short7_finish(const Short7& a, float2 Gc, float2 Gv) {
    const float m1x = a.s1x / a.sw, m1y = a.s1y / a.sw, m2x = a.s2x / a.sw, m2y = a.s2y / a.sw;
    const bool vx = m2x - m1x * m1x > 0.f, vy = m2y - m1y * m1y > 0.f;
    ShortG G;
    G.G1x = Gc.x - (vx ? 2.f * m1x * Gv.x : 0.f);
    G.G1y = Gc.y - (vy ? 2.f * m1y * Gv.y : 0.f);
    G.G2x = vx ? Gv.x : 0.f;
    G.G2y = vy ? Gv.y : 0.f;
    G.c0 = -(G.G1x * m1x + G.G2x * m2x + G.G1y * m1y + G.G2y * m2y);
    G.isw = 1.f / a.sw;
    return G;
}

// dL/d s of tap (dx, dy) of pixel (x, y) into the block's shared tile
// (origin bx0, by0: the block's first pixel minus the apron), and the tap's
// sigma terms dL/d w_q d w_q / d sigma into gsz, gsn (d w / d sigma_z = w
// |dz| a_off / D^2, d w / d sigma_n = w ln(n . n_q))
__device__ __forceinline__ void short7_scatter(const SvgfConsts& k, const float4* g_cur, const float* sig, int N,
                                               float4 zn, float2 gz, int x, int y, int dx, int dy, const ShortG& G,
                                               float (*tile)[kTH][kTW], int bx0, int by0, float& gsz,
                                               float& gsn) {
    using S = Store<DHR_FP32>;
    const int qx = x + dx, qy = y + dy;
    const bool in = qx >= 0 && qy >= 0 && qx < k.W && qy < k.H;
    const long long qi = (long long)min(max(qy, 0), k.H - 1) * k.W + min(max(qx, 0), k.W - 1);
    const int q = (int)dbg_index(qi, (long long)N, kSiteAdjoint);
    const float4 zq = S::g(g_cur, q);
    const float sx = sig[q], sy = sig[N + q];
    if (!in || !is_fg(zq.x)) return;
    const W7 t = w7(k, zn, gz, dx, dy, zq);
    const float w = t.w * G.isw;
    atomicAdd(&tile[0][qy - by0][qx - bx0], (G.G1x + G.G2x * 2.f * sx) * w);
    atomicAdd(&tile[1][qy - by0][qx - bx0], (G.G1y + G.G2y * 2.f * sy) * w);
    if (dx || dy) {
        const float gw = fmaf(sx, fmaf(G.G2x, sx, G.G1x), fmaf(sy, fmaf(G.G2y, sy, G.G1y), G.c0)) * w;
        gsz = fmaf(gw, t.dz * t.a_off * t.rD * t.rD, gsz);
        if (t.nd > 0.f) gsn = fmaf(gw, t.l2n * kLn2, gsn);
    }
}

// A block's 7x7 neighbourhoods staged in shared memory: the G-buffer and
// both signal planes of the kTW x kTH pixels around its tile (outside the
// image: depth +inf, which gives weight exactly 0, and signals 0).
struct ShortStage {
    float4 z[kTH][kTW];
    float2 s[kTH][kTW];
};

// the whole 7x7 estimate of one lane's own pixel (tile position tx, ty),
// its taps read from the staged neighbourhood
__device__ __forceinline__ void short7_lane(const SvgfConsts& k, const ShortStage& st, float4 zn, float2 gz,
                                            int tx, int ty, float2 Gc, float2 Gv, float (*tile)[kTH][kTW],
                                            float& gsz, float& gsn) {
    Short7 a = {};
    for (int dy = -3; dy <= 3; ++dy)
#pragma unroll
        for (int dx = -3; dx <= 3; ++dx) {
            const float4 zq = st.z[ty + kTR + dy][tx + kTR + dx];
            const float2 sq = st.s[ty + kTR + dy][tx + kTR + dx];
            const float w = is_fg(zq.x) ? w7(k, zn, gz, dx, dy, zq).w : 0.f;
            a.sw += w;
            a.s1x = fmaf(w, sq.x, a.s1x);
            a.s1y = fmaf(w, sq.y, a.s1y);
            a.s2x = fmaf(w, sq.x * sq.x, a.s2x);
            a.s2y = fmaf(w, sq.y * sq.y, a.s2y);
        }
    const ShortG G = short7_finish(a, Gc, Gv);
    for (int dy = -3; dy <= 3; ++dy)
#pragma unroll
        for (int dx = -3; dx <= 3; ++dx) {
            const float4 zq = st.z[ty + kTR + dy][tx + kTR + dx];
            const float2 sq = st.s[ty + kTR + dy][tx + kTR + dx];
            if (!is_fg(zq.x)) continue;
            const W7 t = w7(k, zn, gz, dx, dy, zq);
            const float w = t.w * G.isw;
            atomicAdd(&tile[0][ty + kTR + dy][tx + kTR + dx], (G.G1x + G.G2x * 2.f * sq.x) * w);
            atomicAdd(&tile[1][ty + kTR + dy][tx + kTR + dx], (G.G1y + G.G2y * 2.f * sq.y) * w);
            if (dx || dy) {
                const float gw = fmaf(sq.x, fmaf(G.G2x, sq.x, G.G1x), fmaf(sq.y, fmaf(G.G2y, sq.y, G.G1y), G.c0)) * w;
                gsz = fmaf(gw, t.dz * t.a_off * t.rD * t.rD, gsz);
                if (t.nd > 0.f) gsn = fmaf(gw, t.l2n * kLn2, gsn);
            }
        }
}

__global__ void __launch_bounds__(kThreadsA, 4) temporal_bwd_kernel(
    SvgfConsts k, dhr_camera cam, dhr_camera cam_prev, const float4* g_cur, const uint32_t* mesh_cur,
    const float4* g_prev, const uint32_t* mesh_prev, const float* sig, const float4* mom, const uint8_t* hist,
    Upstream up, const float4* gmom, float* g_sig, float2* gcol_prev, float4* gmom_prev, float4* gs) {
    using S = Store<DHR_FP32>;
    __shared__ float tile[2][kTH][kTW];
    __shared__ ShortStage stage;
    const int tid = threadIdx.y * kBX + threadIdx.x, lane = threadIdx.x & 31;
    for (int e = tid; e < 2 * kTH * kTW; e += kThreadsA) (&tile[0][0][0])[e] = 0.f;
    __syncthreads();
    const int bx0 = blockIdx.x * kBX - kTR, by0 = blockIdx.y * kBY - kTR;
    const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
    const int N = k.W * k.H;
    float gsz = 0.f, gsn = 0.f;
    const bool inside = x < k.W && y < k.H;
    const int p = inside ? y * k.W + x : 0;
    const float4 zn = inside ? S::g(g_cur, p) : make_float4(INFINITY, 0.f, 0.f, 0.f);
    const bool fg = inside && is_fg(zn.x);
    int n = 0;
    float2 gz = make_float2(0.f, 0.f), Gc = make_float2(0.f, 0.f), Gv = make_float2(0.f, 0.f);
    float2 Gce = make_float2(0.f, 0.f), s = make_float2(0.f, 0.f);
    float4 Gm = make_float4(0.f, 0.f, 0.f, 0.f);
    float a = 1.0f;
    Reproj r;
    bool valid = false;
    if (fg) {
        n = hist[p];
        gz = depth_grad<S>(g_cur, k.W, k.H, x, y, zn.x);
        if (g_prev && n >= 2) {
            const float slope = fmaxf(fabsf(gz.x), fabsf(gz.y));
            valid = reproject<S>(cam, cam_prev, k.W, k.H, x, y, zn, __ldg(mesh_cur + p), slope, g_prev, mesh_prev, r);
        }
        a = valid ? (k.fixed_alpha ? k.alpha : fmaxf(k.alpha, 1.0f / (float)n)) : 1.0f;
        s = make_float2(sig[p], sig[N + p]);
        Gm = gmom[p];
        const float4 G = upstream(up, N, p);   // at the temporal output (level 0's input)
        Gc = make_float2(G.x, G.y);
        Gv = make_float2(G.z, G.w);
        if (n >= 4) {
            Gce = Gc;
            const float4 m = mom[p];
            if (m.z - m.x * m.x > 0.f) {
                Gm.z += Gv.x;
                Gm.x -= 2.f * m.x * Gv.x;
            }
            if (m.w - m.y * m.y > 0.f) {
                Gm.w += Gv.y;
                Gm.y -= 2.f * m.y * Gv.y;
            }
        }
    }
    // short history (n < 4): backward of the 7x7 spatial estimate.  A warp
    // with many such lanes lets each do its own 49 taps twice (sums, then
    // scatter) on the block's staged neighbourhood; with few, the warp serves
    // them one after another, lane l taking taps l and l + 32, the sums
    // reduced across the warp.
    const bool need = fg && n < 4;
    unsigned todo = __ballot_sync(kFull, need);
    const bool many = __popc(todo) >= kShortPerLane;
    if (__syncthreads_or(many && need)) {   // some warp of the block works per lane: stage
        for (int e = tid; e < kTH * kTW; e += kThreadsA) {
            const int sy = e / kTW, sx = e - sy * kTW;
            const int qx = bx0 + sx, qy = by0 + sy;
            float4 z = make_float4(INFINITY, 0.f, 0.f, 0.f);
            float2 v = make_float2(0.f, 0.f);
            if (qx >= 0 && qy >= 0 && qx < k.W && qy < k.H) {
                const int q = (int)dbg_index((long long)qy * k.W + qx, (long long)N, kSiteAdjoint);
                z = S::g(g_cur, q);
                v = make_float2(sig[q], sig[N + q]);
            }
            stage.z[sy][sx] = z;
            stage.s[sy][sx] = v;
        }
        __syncthreads();
    }
    if (many) {
        if (need) short7_lane(k, stage, zn, gz, threadIdx.x, threadIdx.y, Gc, Gv, tile, gsz, gsn);
    } else {
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int px = __shfl_sync(kFull, x, src), py = __shfl_sync(kFull, y, src);
            const float4 pz = make_float4(__shfl_sync(kFull, zn.x, src), __shfl_sync(kFull, zn.y, src),
                                          __shfl_sync(kFull, zn.z, src), __shfl_sync(kFull, zn.w, src));
            const float2 pg = make_float2(__shfl_sync(kFull, gz.x, src), __shfl_sync(kFull, gz.y, src));
            const float2 pc = make_float2(__shfl_sync(kFull, Gc.x, src), __shfl_sync(kFull, Gc.y, src));
            const float2 pv = make_float2(__shfl_sync(kFull, Gv.x, src), __shfl_sync(kFull, Gv.y, src));
            Short7 acc = {};
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int t = lane + 32 * it;
                if (t < 49) short7_tap(k, g_cur, sig, N, pz, pg, px, py, t % 7 - 3, t / 7 - 3, acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc.sw += __shfl_xor_sync(kFull, acc.sw, o);
                acc.s1x += __shfl_xor_sync(kFull, acc.s1x, o);
                acc.s1y += __shfl_xor_sync(kFull, acc.s1y, o);
                acc.s2x += __shfl_xor_sync(kFull, acc.s2x, o);
                acc.s2y += __shfl_xor_sync(kFull, acc.s2y, o);
            }
            const ShortG G = short7_finish(acc, pc, pv);
            float dz_s = 0.f, dn_s = 0.f;
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int t = lane + 32 * it;
                if (t < 49)
                    short7_scatter(k, g_cur, sig, N, pz, pg, px, py, t % 7 - 3, t / 7 - 3, G, tile, bx0, by0,
                                         dz_s, dn_s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dz_s += __shfl_xor_sync(kFull, dz_s, o);
                dn_s += __shfl_xor_sync(kFull, dn_s, o);
            }
            if (lane == src) {
                gsz += dz_s;
                gsn += dn_s;
            }
        }
    }
    if (fg) {
        // moving averages
        atomicAdd(&tile[0][y - by0][x - bx0], a * Gce.x + a * Gm.x + 2.f * a * s.x * Gm.z);
        atomicAdd(&tile[1][y - by0][x - bx0], a * Gce.y + a * Gm.y + 2.f * a * s.y * Gm.w);
        if (valid) {
            const float b = 1.f - a;
            for (int t = 0; t < 4; ++t) {
                if (!(r.ok & (1 << t))) continue;
                const int q = (int)dbg_index((long long)(r.y0 + (t >> 1)) * k.W + (r.x0 + (t & 1)), (long long)N,
                                             kSiteAdjoint);
                const float bb = r.w[t] / r.sumw * b;
                atomicAdd(gcol_prev + q, make_float2(bb * Gce.x, bb * Gce.y));
                atomicAdd(gmom_prev + q, make_float4(bb * Gm.x, bb * Gm.y, bb * Gm.z, bb * Gm.w));
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < 2 * kTH * kTW; e += kThreadsA) {
        const int c = e / (kTH * kTW), rr = e % (kTH * kTW);
        const int qx = bx0 + rr % kTW, qy = by0 + rr / kTW;
        const float v = tile[c][rr / kTW][rr % kTW];
        if (v != 0.f && qx >= 0 && qy >= 0 && qx < k.W && qy < k.H) atomicAdd(g_sig + (size_t)c * N + qy * k.W + qx, v);
    }
    if (inside && (gsz != 0.f || gsn != 0.f)) {
        float4 acc = gs[p];
        acc.x += gsz;
        acc.y += gsn;
        gs[p] = acc;
    }
}

// per-block sums (double, then rounded to float) of the per-pixel sigma
// terms: block b sums a fixed contiguous range of pixels in a fixed order
constexpr int kPixReduceBlocks = 296, kPixReduceThreads = 256;
__global__ void __launch_bounds__(kPixReduceThreads) reduce_pixels_kernel(int n, const float4* gs, float* partial) {
    __shared__ double sh[3][kPixReduceThreads];
    const int t = threadIdx.x;
    const int per = (n + gridDim.x - 1) / gridDim.x, b0 = blockIdx.x * per, b1 = min(n, b0 + per);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = b0 + t; i < b1; i += kPixReduceThreads) {
        const float4 v = gs[i];
        s0 += (double)v.x;
        s1 += (double)v.y;
        s2 += (double)v.z;
    }
    sh[0][t] = s0;
    sh[1][t] = s1;
    sh[2][t] = s2;
    __syncthreads();
    for (int o = kPixReduceThreads / 2; o > 0; o >>= 1) {
        if (t < o) {
            sh[0][t] += sh[0][t + o];
            sh[1][t] += sh[1][t + o];
            sh[2][t] += sh[2][t + o];
        }
        __syncthreads();
    }
    if (t < 3) partial[3 * blockIdx.x + t] = (float)sh[t][0];
}

// sum the per-block partials into acc[3] (double) with one block of
// kReduceThreads threads: a fixed assignment of partials to threads and a
// fixed tree, so the sum is the same on every run
constexpr int kReduceThreads = 256;
__global__ void __launch_bounds__(kReduceThreads) reduce_partials_kernel(int nblocks, const float* partial,
                                                                         double* acc) {
    __shared__ double sh[3][kReduceThreads];
    const int t = threadIdx.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = t; b < nblocks; b += kReduceThreads) {
        s0 += (double)partial[3 * b + 0];
        s1 += (double)partial[3 * b + 1];
        s2 += (double)partial[3 * b + 2];
    }
    sh[0][t] = s0;
    sh[1][t] = s1;
    sh[2][t] = s2;
    __syncthreads();
    for (int o = kReduceThreads / 2; o > 0; o >>= 1) {
        if (t < o) {
            sh[0][t] += sh[0][t + o];
            sh[1][t] += sh[1][t + o];
            sh[2][t] += sh[2][t + o];
        }
        __syncthreads();
    }
    if (t < 3) acc[t] += sh[t][0];
}

__global__ void finish_sigma_kernel(const double* acc, float* out) {
    const int c = threadIdx.x;
    if (c < 3) out[c] = (float)acc[c];
}

}  // namespace
}  // namespace dhr

struct dhr_svgf_tape {
    int W = 0, H = 0, F = 0;
    int frames_recorded = 0;
    int levels_recorded = 0;
    float4* illum = nullptr;   // [F][N] temporal outputs
    float4* mom = nullptr;     // [F][N] moments
    uint8_t* hist = nullptr;   // [F][N] history lengths
    float2* col = nullptr;     // [N] colour history (forward)
    float4* lev[2] = {nullptr, nullptr};
    // level records, allocated for `rec_levels` levels and `rec_slots` frames
    // on first use: one slot per frame when the forward stores every frame's
    // levels (DHR_TAPE_STORE); otherwise (DHR_TAPE_RECOMPUTE) two slots, frame
    // f in slot f & 1: the forward leaves the last two frames' records there
    // and the backward recomputes frame f - 1's levels on `side` while frame
    // f's adjoint runs
    float4* lvs = nullptr;     // [slots][levels - 1][N] inputs of levels 1..
    float2* wsum = nullptr;    // [slots][levels][N] weight sums of every level
    float4* last = nullptr;    // [slots][N] filtered colour and variance of the last level
    int rec_levels = 0;
    int rec_slots = 0;
    int schedule = DHR_TAPE_RECOMPUTE;
    int slot_frame[2] = {-1, -1};   // DHR_TAPE_RECOMPUTE: the frame whose records a slot holds
    // DHR_TAPE_RECOMPUTE: the backward's passes run on `mainq` (highest
    // priority), the recomputation on `side` (lowest), so that recompute blocks
    // take only the SM slots the passes leave free
    cudaStream_t side = nullptr, mainq = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_main = nullptr, ev_ready[2] = {nullptr, nullptr},
                ev_free[2] = {nullptr, nullptr};
    float2* gcol[2] = {nullptr, nullptr};
    float4* gmom[2] = {nullptr, nullptr};
    float2* gc = nullptr;      // [N] dL/d colour at the input of the level just processed
    float2* gv = nullptr;      // [N] dL/d variance, same
    float4* rec = nullptr;     // [4][N] pass-A records
    float4* gs = nullptr;      // [N] per-pixel (dL/d sigma_z, dL/d sigma_n, dL/d sigma_l, -)
    float* partial = nullptr;  // [kPixReduceBlocks][3]
    double* acc = nullptr;     // [3]
    int nblocks = 0;
};

// levels the differentiable form accepts (check_svgf_params enforces it)
constexpr int kMaxLevels = 8;

using namespace dhr;

static void tape_free(dhr_svgf_tape* t) {
    if (!t) return;
    cudaFree(t->illum);
    cudaFree(t->mom);
    cudaFree(t->hist);
    cudaFree(t->col);
    for (int i = 0; i < 2; ++i) {
        cudaFree(t->lev[i]);
        cudaFree(t->gcol[i]);
        cudaFree(t->gmom[i]);
    }
    cudaFree(t->gc);
    cudaFree(t->gv);
    cudaFree(t->rec);
    cudaFree(t->gs);
    cudaFree(t->lvs);
    cudaFree(t->wsum);
    cudaFree(t->last);
    cudaFree(t->partial);
    cudaFree(t->acc);
    for (cudaEvent_t e : {t->ev_fork, t->ev_join, t->ev_main, t->ev_ready[0], t->ev_ready[1], t->ev_free[0],
                          t->ev_free[1]})
        if (e) cudaEventDestroy(e);
    if (t->side) cudaStreamDestroy(t->side);
    if (t->mainq) cudaStreamDestroy(t->mainq);
    delete t;
}

extern "C" void dhr_svgf_tape_destroy(dhr_svgf_tape* tape) { tape_free(tape); }

extern "C" dhr_status dhr_svgf_tape_create(int32_t width, int32_t height, int32_t frames, dhr_svgf_tape** out) {
    clear_error();
    DHR_CHECK_ARG(out, "svgf_tape_create: null out");
    DHR_CHECK_ARG(width > 0 && height > 0 && (int64_t)width * height <= (1ll << 27) && frames >= 1 && frames <= 1024,
                  "svgf_tape_create: bad size %dx%d x %d frames", width, height, frames);
    auto* t = new dhr_svgf_tape();
    t->W = width;
    t->H = height;
    t->F = frames;
    const size_t n = (size_t)width * height;
    const dim3 grid((width + kBX - 1) / kBX, (height + kBY - 1) / kBY);
    t->nblocks = (int)(grid.x * grid.y);
    cudaError_t e = cudaMalloc((void**)&t->illum, (size_t)frames * n * 16);
    if (!e) e = cudaMalloc((void**)&t->mom, (size_t)frames * n * 16);
    if (!e) e = cudaMalloc((void**)&t->hist, (size_t)frames * n);
    if (!e) e = cudaMalloc((void**)&t->col, n * 8);
    for (int i = 0; i < 2 && !e; ++i) {
        e = cudaMalloc((void**)&t->lev[i], n * 16);
        if (!e) e = cudaMalloc((void**)&t->gcol[i], n * 8);
        if (!e) e = cudaMalloc((void**)&t->gmom[i], n * 16);
    }
    if (!e) e = cudaMalloc((void**)&t->gc, n * 8);
    if (!e) e = cudaMalloc((void**)&t->gv, n * 8);
    if (!e) e = cudaMalloc((void**)&t->rec, n * 64);
    if (!e) e = cudaMalloc((void**)&t->gs, n * 16);
    if (!e) e = cudaMalloc((void**)&t->partial, (size_t)kPixReduceBlocks * 3 * sizeof(float));
    if (!e) e = cudaMalloc((void**)&t->acc, 3 * sizeof(double));
    int least = 0, greatest = 0;
    if (!e) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (!e) e = cudaStreamCreateWithPriority(&t->side, cudaStreamNonBlocking, least);
    if (!e) e = cudaStreamCreateWithPriority(&t->mainq, cudaStreamNonBlocking, greatest);
    for (cudaEvent_t* ev : {&t->ev_fork, &t->ev_join, &t->ev_main, &t->ev_ready[0], &t->ev_ready[1],
                            &t->ev_free[0], &t->ev_free[1]})
        if (!e) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e) {
        cudaGetLastError();
        tape_free(t);
        return set_error(e == cudaErrorMemoryAllocation ? DHR_ERR_OOM : DHR_ERR_CUDA, "svgf_tape_create: %s",
                         cudaGetErrorString(e));
    }
    *out = t;
    return DHR_OK;
}

static dhr_status check_seq(const dhr_svgf_tape* t, const dhr_gbuffer* g, const dhr_camera* cams,
                            const dhr_svgf_params* p) {
    DHR_CHECK_ARG(t && g && cams && p, "svgf_seq: null pointer");
    DHR_TRY(check_svgf_params(p));
    DHR_CHECK_ARG(atrous_radius(p) == 2, "svgf_seq: the differentiable form takes the 5x5 kernel only");
    for (int f = 0; f < t->F; ++f) {
        DHR_CHECK_ARG(g[f].precision == DHR_FP32, "svgf_seq: the differentiable form runs on FP32 G-buffers");
        DHR_CHECK_ARG(g[f].width == t->W && g[f].height == t->H && g[f].depth_normal && g[f].mesh_id &&
                          cams[f].width == t->W && cams[f].height == t->H,
                      "svgf_seq: frame %d does not match the tape (%dx%d)", f, t->W, t->H);
    }
    return DHR_OK;
}

// Level records of one frame in slot `slot`: input of level l (l >= 1),
// output of level l, weight sums of level l.
struct LevelSlot {
    const dhr_svgf_tape* t;
    size_t N;
    int L, slot;
    float4* in(int l, const float4* illum) const {
        return l == 0 ? const_cast<float4*>(illum) : t->lvs + ((size_t)slot * (L - 1) + (l - 1)) * N;
    }
    float4* out(int l) const {
        return l + 1 < L ? t->lvs + ((size_t)slot * (L - 1) + l) * N : t->last + (size_t)slot * N;
    }
    float2* wsum(int l) const { return t->wsum + ((size_t)slot * L + l) * N; }
};

static int level_slots(const dhr_svgf_tape* t) {
    return t->schedule == DHR_TAPE_STORE ? t->F : (t->F < 2 ? t->F : 2);
}

static dhr_status alloc_level_records(dhr_svgf_tape* t, int L, size_t N) {
    const int slots = level_slots(t);
    if (L <= t->rec_levels && slots == t->rec_slots) return DHR_OK;
    cudaFree(t->lvs);
    cudaFree(t->wsum);
    cudaFree(t->last);
    t->lvs = nullptr;
    t->wsum = nullptr;
    t->last = nullptr;
    t->rec_levels = 0;
    t->rec_slots = 0;
    t->slot_frame[0] = t->slot_frame[1] = -1;
    cudaError_t e = cudaSuccess;
    if (L > 1) e = cudaMalloc((void**)&t->lvs, (size_t)slots * (L - 1) * N * 16);
    if (!e) e = cudaMalloc((void**)&t->wsum, (size_t)slots * L * N * 8);
    if (!e) e = cudaMalloc((void**)&t->last, (size_t)slots * N * 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? DHR_ERR_OOM : DHR_ERR_CUDA,
                         "svgf_seq_forward: level records: %s", cudaGetErrorString(e));
    }
    t->rec_levels = L;
    t->rec_slots = slots;
    return DHR_OK;
}

// The L recorded a-trous levels of one frame (Section 3.3's filter with the
// weight sums kept): level 0 writes the colour history `col`, the last level
// (L >= 2) the planes ao / sh; with L == 1 the single level's output is the
// slot's last-level record.  col == nullptr: the records only (a recompute).
static dhr_status run_levels(const SvgfConsts& k, int nsq, cudaStream_t st, const float4* g, const float4* illum,
                             const LevelSlot& s, float2* col, float* ao, float* sh) {
    for (int l = 0; l < s.L; ++l) {
        const int mode = (l == s.L - 1 && s.L > 1) ? 2 : (l == 0 && col ? 1 : 0);
        DHR_TRY(launch_atrous_recorded(mode, nsq, st, k, 1 << l, g, s.in(l, illum), s.out(l), col, ao, sh,
                                       AtrousRec{s.wsum(l), s.t->last + (size_t)s.slot * s.N}));
    }
    return DHR_OK;
}

extern "C" dhr_status dhr_svgf_tape_set_schedule(dhr_svgf_tape* t, int32_t schedule) {
    clear_error();
    DHR_CHECK_ARG(t, "svgf_tape_set_schedule: null tape");
    DHR_CHECK_ARG(schedule == DHR_TAPE_RECOMPUTE || schedule == DHR_TAPE_STORE,
                  "svgf_tape_set_schedule: unknown schedule %d", schedule);
    if (schedule != t->schedule) {
        t->schedule = schedule;
        t->frames_recorded = 0;   // the records of the last forward no longer fit the schedule
        t->slot_frame[0] = t->slot_frame[1] = -1;
    }
    return DHR_OK;
}

extern "C" dhr_status dhr_svgf_tape_level_bytes(const dhr_svgf_tape* t, int32_t levels, int64_t* bytes) {
    clear_error();
    DHR_CHECK_ARG(t && bytes, "svgf_tape_level_bytes: null pointer");
    DHR_CHECK_ARG(levels >= 0 && levels <= kMaxLevels, "svgf_tape_level_bytes: levels %d outside 0..%d", levels,
                  kMaxLevels);
    const int64_t N = (int64_t)t->W * t->H, slots = level_slots(t);
    *bytes = levels == 0 ? 0 : slots * N * (16 * (levels - 1) + 8 * levels + 16);
    return DHR_OK;
}

extern "C" dhr_status dhr_svgf_seq_forward(dhr_svgf_tape* t, const dhr_gbuffer* gbufs, const dhr_camera* cams,
                                           const float* sig, const dhr_svgf_params* params, float* out,
                                           void* stream) {
    clear_error();
    DHR_TRY(check_seq(t, gbufs, cams, params));
    DHR_CHECK_ARG(sig && out, "svgf_seq_forward: null signal or output");
    cudaStream_t st = as_stream(stream);
    using S = Store<DHR_FP32>;
    const SvgfConsts k = make_consts(t->W, t->H, params);
    const int nsq = atrous_nsq(params);
    const size_t N = (size_t)t->W * t->H;
    const dim3 blk(32, 8), grid((t->W + 31) / 32, (t->H + 7) / 8);
    const int L = (int)params->levels;
    DHR_CHECK_ARG(L <= kMaxLevels, "svgf_seq_forward: levels %d > %d", L, kMaxLevels);
    t->frames_recorded = 0;
    t->slot_frame[0] = t->slot_frame[1] = -1;
    if (L > 0) DHR_TRY(alloc_level_records(t, L, N));
    const bool store = t->schedule == DHR_TAPE_STORE;
    for (int f = 0; f < t->F; ++f) {
        const bool hp = f > 0;
        const auto* gc = static_cast<const S::G*>(gbufs[f].depth_normal);
        const auto* gp = hp ? static_cast<const S::G*>(gbufs[f - 1].depth_normal) : nullptr;
        float4* illum = t->illum + (size_t)f * N;
        temporal_kernel<DHR_FP32, SigPlanar><<<grid, blk, 0, st>>>(
            k, cams[f], hp ? cams[f - 1] : cams[f], gc, gbufs[f].mesh_id, gp, hp ? gbufs[f - 1].mesh_id : nullptr,
            SigPlanar{sig + (size_t)f * 2 * N, N}, t->col, hp ? t->mom + (size_t)(f - 1) * N : t->mom,
            hp ? t->hist + (size_t)(f - 1) * N : t->hist, t->mom + (size_t)f * N, t->hist + (size_t)f * N, illum);
        DHR_CUDA_TRY(cudaGetLastError());
        float* ao = out + (size_t)f * 2 * N;
        float* sh = ao + N;
        if (L == 0) {
            passthrough_kernel<DHR_FP32><<<(int)((N + 255) / 256), 256, 0, st>>>((int)N, illum, t->col, ao, sh);
            DHR_CUDA_TRY(cudaGetLastError());
            continue;
        }
        const float4* last_out;
        if (store || f + 2 >= t->F) {   // records kept: every frame, or the last two
            const LevelSlot s{t, N, L, store ? f : (f & 1)};
            DHR_TRY(run_levels(k, nsq, st, gc, illum, s, t->col, ao, sh));
            last_out = s.out(0);
        } else {   // the backward recomputes this frame's records: plain levels
            const float4* in = illum;
            for (int l = 0; l < L; ++l) {
                const int mode = (l == L - 1 && L > 1) ? 2 : (l == 0 ? 1 : 0);
                DHR_TRY(launch_atrous<DHR_FP32>(mode, nsq, 2, st, k, 1 << l, gc, in, t->lev[l & 1], t->col, ao, sh));
                in = t->lev[l & 1];
            }
            last_out = t->lev[0];
        }
        if (L == 1) {
            passthrough_kernel<DHR_FP32><<<(int)((N + 255) / 256), 256, 0, st>>>((int)N, last_out, t->col, ao, sh);
            DHR_CUDA_TRY(cudaGetLastError());
        }
    }
    t->frames_recorded = t->F;
    t->levels_recorded = L;
    if (!store && L > 0)
        for (int f = t->F - 1; f >= 0 && f >= t->F - 2; --f) t->slot_frame[f & 1] = f;
    return DHR_OK;
}

extern "C" dhr_status dhr_svgf_seq_backward(dhr_svgf_tape* t, const dhr_gbuffer* gbufs, const dhr_camera* cams,
                                            const float* sig, const dhr_svgf_params* params, const float* g_out,
                                            float* g_sig, float* g_sigma, void* stream) {
    clear_error();
    DHR_TRY(check_seq(t, gbufs, cams, params));
    DHR_CHECK_ARG(sig && g_out && g_sig && g_sigma, "svgf_seq_backward: null pointer");
    if (t->frames_recorded != t->F)
        return set_error(DHR_ERR_STATE, "svgf_seq_backward: run dhr_svgf_seq_forward on this tape first");
    if (t->levels_recorded != (int)params->levels)
        return set_error(DHR_ERR_STATE, "svgf_seq_backward: the forward ran %d levels, not %d", t->levels_recorded,
                         (int)params->levels);
    cudaStream_t st = as_stream(stream);
    using S = Store<DHR_FP32>;
    const SvgfConsts k = make_consts(t->W, t->H, params);
    const int nsq = atrous_nsq(params);
    const size_t N = (size_t)t->W * t->H;
    const int n = (int)N;
    const dim3 blk(32, 8), grid((t->W + 31) / 32, (t->H + 7) / 8);
    const int L = (int)params->levels;
    const bool store = t->schedule == DHR_TAPE_STORE;
    DHR_CUDA_TRY(cudaMemsetAsync(g_sig, 0, (size_t)t->F * 2 * N * sizeof(float), st));
    DHR_CUDA_TRY(cudaMemsetAsync(t->gs, 0, N * 16, st));
    DHR_CUDA_TRY(cudaMemsetAsync(t->acc, 0, 3 * sizeof(double), st));
    DHR_CUDA_TRY(cudaMemsetAsync(t->gcol[0], 0, N * 8, st));
    DHR_CUDA_TRY(cudaMemsetAsync(t->gmom[0], 0, N * 16, st));
    // DHR_TAPE_RECOMPUTE: frame f's records are in slot f & 1; a frame the
    // slots do not hold is recomputed on the side stream one frame ahead,
    // into the slot frame f + 1's adjoint has finished with
    const bool side = L > 0 && !store;
    cudaStream_t ms = side ? t->mainq : st;   // the passes' stream
    bool pending[2] = {false, false};
    auto prefetch = [&](int f) -> dhr_status {
        const int sl = f & 1;
        if (t->slot_frame[sl] == f) return DHR_OK;
        t->slot_frame[sl] = -1;
        if (f + 2 < t->F) DHR_CUDA_TRY(cudaStreamWaitEvent(t->side, t->ev_free[sl], 0));
        DHR_TRY(run_levels(k, nsq, t->side, static_cast<const S::G*>(gbufs[f].depth_normal), t->illum + (size_t)f * N,
                           LevelSlot{t, N, L, sl}, nullptr, nullptr, nullptr));
        DHR_CUDA_TRY(cudaEventRecord(t->ev_ready[sl], t->side));
        pending[sl] = true;
        t->slot_frame[sl] = f;
        return DHR_OK;
    };
    auto frames = [&]() -> dhr_status {
        if (side) DHR_TRY(prefetch(t->F - 1));
        int nx = 0;   // index of the "from the next frame" gradient buffers
        for (int f = t->F - 1; f >= 0; --f) {
            const auto* gcur = static_cast<const S::G*>(gbufs[f].depth_normal);
            const float4* illum = t->illum + (size_t)f * N;
            const LevelSlot s{t, N, L, store ? f : (f & 1)};
            if (side && f > 0) DHR_TRY(prefetch(f - 1));
            if (side && pending[f & 1]) {
                DHR_CUDA_TRY(cudaStreamWaitEvent(ms, t->ev_ready[f & 1], 0));
                pending[f & 1] = false;
            }
            // the gradient at the output of the level being processed comes
            // from the loss (last level) or from pass B of the level above
            Upstream up{g_out + (size_t)f * 2 * N, nullptr, nullptr, L <= 1 ? t->gcol[nx] : nullptr};
            for (int l = L - 1; l >= 0; --l) {
                const float4* xin = s.in(l, illum);
                const float4* xout = s.out(l);
                const float2* ws = s.wsum(l);
                if (nsq == 7 && k.wl_in_atrous)
                    atrous_bwd_a<7, true><<<grid, blk, 0, ms>>>(k, 1 << l, gcur, xin, ws, xout, up, t->rec, t->gs);
                else if (nsq == 7)
                    atrous_bwd_a<7, false><<<grid, blk, 0, ms>>>(k, 1 << l, gcur, xin, ws, xout, up, t->rec, t->gs);
                else if (k.wl_in_atrous)
                    atrous_bwd_a<-1, true><<<grid, blk, 0, ms>>>(k, 1 << l, gcur, xin, ws, xout, up, t->rec, t->gs);
                else
                    atrous_bwd_a<-1, false><<<grid, blk, 0, ms>>>(k, 1 << l, gcur, xin, ws, xout, up, t->rec,
                                                                  t->gs);
                DHR_CUDA_TRY(cudaGetLastError());
                if (nsq == 7)
                    atrous_bwd_b<7><<<grid, blk, 0, ms>>>(k, 1 << l, gcur, xin, t->rec, t->gc, t->gv);
                else
                    atrous_bwd_b<-1><<<grid, blk, 0, ms>>>(k, 1 << l, gcur, xin, t->rec, t->gc, t->gv);
                DHR_CUDA_TRY(cudaGetLastError());
                // level l - 1's output gradient (plus, for level 0's output,
                // the next frame's colour-history gradient)
                up = Upstream{nullptr, t->gc, t->gv, l == 1 ? t->gcol[nx] : nullptr};
            }
            if (side) DHR_CUDA_TRY(cudaEventRecord(t->ev_free[f & 1], ms));   // slot f & 1 read for the last time
            const int pv = nx ^ 1;
            DHR_CUDA_TRY(cudaMemsetAsync(t->gcol[pv], 0, N * 8, ms));
            DHR_CUDA_TRY(cudaMemsetAsync(t->gmom[pv], 0, N * 16, ms));
            const bool hp = f > 0;
            // at the temporal output: pass B of level 0, or the loss gradient
            // plus the colour-history gradient when there are no levels
            up.gcol = L == 0 ? t->gcol[nx] : nullptr;
            temporal_bwd_kernel<<<grid, blk, 0, ms>>>(
                k, cams[f], hp ? cams[f - 1] : cams[f], gcur, gbufs[f].mesh_id,
                hp ? static_cast<const S::G*>(gbufs[f - 1].depth_normal) : nullptr,
                hp ? gbufs[f - 1].mesh_id : nullptr, sig + (size_t)f * 2 * N, t->mom + (size_t)f * N,
                t->hist + (size_t)f * N, up, t->gmom[nx], g_sig + (size_t)f * 2 * N, t->gcol[pv], t->gmom[pv],
                t->gs);
            DHR_CUDA_TRY(cudaGetLastError());
            nx = pv;
        }
        return DHR_OK;
    };
    if (side) {   // both tape streams start after everything before this call on `st`
        DHR_CUDA_TRY(cudaEventRecord(t->ev_fork, st));
        DHR_CUDA_TRY(cudaStreamWaitEvent(t->side, t->ev_fork, 0));
        DHR_CUDA_TRY(cudaStreamWaitEvent(t->mainq, t->ev_fork, 0));
    }
    const dhr_status r = frames();
    if (side) {   // and `st` continues after all of their work, also on an error
        cudaError_t e2 = cudaEventRecord(t->ev_join, t->side);
        if (!e2) e2 = cudaEventRecord(t->ev_main, t->mainq);
        if (!e2) e2 = cudaStreamWaitEvent(st, t->ev_join, 0);
        if (!e2) e2 = cudaStreamWaitEvent(st, t->ev_main, 0);
        if (r != DHR_OK || e2) t->slot_frame[0] = t->slot_frame[1] = -1;
        if (r != DHR_OK) return r;
        DHR_CUDA_TRY(e2);
    }
    if (r != DHR_OK) return r;
    reduce_pixels_kernel<<<kPixReduceBlocks, kPixReduceThreads, 0, st>>>(n, t->gs, t->partial);
    DHR_CUDA_TRY(cudaGetLastError());
    reduce_partials_kernel<<<1, kReduceThreads, 0, st>>>(kPixReduceBlocks, t->partial, t->acc);
    DHR_CUDA_TRY(cudaGetLastError());
    finish_sigma_kernel<<<1, 32, 0, st>>>(t->acc, g_sigma);
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}
