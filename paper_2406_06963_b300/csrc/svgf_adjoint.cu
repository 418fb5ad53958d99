// Adjoint of the modified SVGF (Section 3.3) over a sequence of frames.
//
// The paper has no gradient; this is the differentiable form of its filter:
// a loss on the filtered colour is back-propagated to the per-pixel noisy
// signals (AO, shadow) of every frame and to the edge-stopping parameters
// sigma_z, sigma_n, sigma_l, through all a-trous levels, the variance
// estimate, the moving averages and the reprojected history of earlier
// frames (the temporal recursion is not cut).
//
// Forward (dhr_svgf_seq_forward) records per frame only the temporal output
// (colour, variance), the moments and the history lengths; the a-trous
// levels are recomputed during the backward pass.  Backward of one a-trous
// level is a two-pass gather:
//   pass A (per output pixel p): re-evaluate the level at p and form the
//     per-pixel factors of dL/dw_pq = a1 c_q - a2 + a3 w_pq v_q, the
//     gradient through p's own colour and p's luminance scale;
//   pass B (per input pixel q): gather from the 25 pixels whose footprint
//     contains q (and the 9 whose variance Gaussian does).
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

// block sum of three values into out[blockIdx linear][3]
__device__ __forceinline__ void block_sum3(float a, float b, float c, float* out) {
    __shared__ float sh[3][kThreadsA / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(kFull, a, o);
        b += __shfl_xor_sync(kFull, b, o);
        c += __shfl_xor_sync(kFull, c, o);
    }
    const int t = threadIdx.y * blockDim.x + threadIdx.x, w = t >> 5;
    if ((t & 31) == 0) {
        sh[0][w] = a;
        sh[1][w] = b;
        sh[2][w] = c;
    }
    __syncthreads();
    if (t == 0) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int i = 0; i < kThreadsA / 32; ++i) {
            s0 += sh[0][i];
            s1 += sh[1][i];
            s2 += sh[2][i];
        }
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        out[3 * blk + 0] = s0;
        out[3 * blk + 1] = s1;
        out[3 * blk + 2] = s2;
    }
}

// Weight of tap q for output pixel p at offset (i, j) * step, per channel,
// with the factors needed by the derivatives.
struct TapW {
    float w0, w1;     // full weights
    float a_off;      // |grad z_p . (p - q)|
    float D;          // sigma_z a_off + eps_z
    float dz;         // |z_p - z_q|
    float nd;         // n_p . n_q
};

// The weight is evaluated as one power of two, as in the forward kernel:
// 2^(log2(h_i h_j) + sigma_n log2(n.n_q) - log2(e) (|dz| / D + |dc| il)).
template <int kNsq>
__device__ __forceinline__ TapW tap_weight(const SvgfConsts& k, int step, int i, int j, float4 zp, float2 gz,
                                           float cp0, float cp1, float il0, float il1, float4 zq, float cq0,
                                           float cq1) {
    const float l5[5] = {-4.f, -2.f, -1.41503750f, -2.f, -4.f};
    TapW t;
    t.a_off = (float)step * fabsf(fmaf(gz.x, (float)i, gz.y * (float)j));
    t.D = fmaf(k.sigma_z, t.a_off, k.eps_z);
    t.dz = fabsf(zp.x - zq.x);
    t.nd = zp.y * zq.y + zp.z * zq.z + zp.w * zq.w;
    const float e = fmaf(-kLog2e, t.dz * rcp_approx(t.D), l5[i + 2] + l5[j + 2]) + log2_normal<kNsq>(t.nd, k.sigma_n);
    t.w0 = ex2_approx(fmaf(-kLog2e * il0, fabsf(cp0 - cq0), e));
    t.w1 = ex2_approx(fmaf(-kLog2e * il1, fabsf(cp1 - cq1), e));
    return t;
}

// records of pass A, 4 x float4 per pixel:
//   r0 = (a1, a2, a3, il) of channel 0, r1 = same for channel 1,
//   r2 = (Gg0, Gg1, self0, self1), r3 = (gz.x, gz.y, -, -)
// Gg already divided by the pixel's Gaussian normaliser.
template <int kNsq>
__global__ void __launch_bounds__(kThreadsA) atrous_bwd_a(SvgfConsts k, int step, const float4* g, const float4* x,
                                                          const float2* gc, const float2* gv, float4* rec,
                                                          float* partial) {
    using S = Store<DHR_FP32>;
    const int px = blockIdx.x * kBX + threadIdx.x, py = blockIdx.y * kBY + threadIdx.y;
    float gsz = 0.f, gsn = 0.f, gsl = 0.f;
    const bool inside = px < k.W && py < k.H;
    const int p = inside ? py * k.W + px : 0;
    float4 cp = make_float4(0.f, 0.f, -1.f, -1.f);
    if (inside) cp = __ldg(x + p);
    if (inside && fg_var(cp.z)) {
        const float4 zp = S::g(g, p);
        float gv0 = 0.f, gv1 = 0.f, gw = 0.f;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int qx = px + dx, qy = py + dy;
                if (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H) continue;
                const float4 v = __ldg(x + qy * k.W + qx);
                if (!fg_var(v.z)) continue;
                const float kk = (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f);
                gw += kk;
                gv0 = fmaf(kk, v.z, gv0);
                gv1 = fmaf(kk, v.w, gv1);
            }
        const float root0 = sqrtf(fmaxf(0.f, gv0 / gw)), root1 = sqrtf(fmaxf(0.f, gv1 / gw));
        const float il0 = k.wl_in_atrous ? 1.0f / (k.sigma_l * root0 + k.eps_l) : 0.f;
        const float il1 = k.wl_in_atrous ? 1.0f / (k.sigma_l * root1 + k.eps_l) : 0.f;
        const float2 gz = depth_grad<S>(g, k.W, k.H, px, py, zp.x);
        const float kc = 0.375f * 0.375f;
        // pass 1: W, A, B per channel
        float W0 = kc, W1 = kc, A0 = kc * cp.x, A1 = kc * cp.y, B0 = kc * kc * cp.z, B1 = kc * kc * cp.w;
        for (int j = -2; j <= 2; ++j)
            for (int i = -2; i <= 2; ++i) {
                if (!i && !j) continue;
                const int qx = px + i * step, qy = py + j * step;
                if (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H) continue;
                const int q = qy * k.W + qx;
                const float4 cq = __ldg(x + q);
                if (!fg_var(cq.z)) continue;
                const TapW t = tap_weight<kNsq>(k, step, i, j, zp, gz, cp.x, cp.y, il0, il1, S::g(g, q), cq.x, cq.y);
                W0 += t.w0;
                W1 += t.w1;
                A0 = fmaf(t.w0, cq.x, A0);
                A1 = fmaf(t.w1, cq.y, A1);
                B0 = fmaf(t.w0 * t.w0, cq.z, B0);
                B1 = fmaf(t.w1 * t.w1, cq.w, B1);
            }
        const float c0 = A0 / W0, c1 = A1 / W1, v0 = B0 / (W0 * W0), v1 = B1 / (W1 * W1);
        const float2 Gc = gc[p], Gv = gv[p];
        const float a10 = Gc.x / W0, a11 = Gc.y / W1;
        const float a20 = (Gc.x * c0 + 2.f * Gv.x * v0) / W0, a21 = (Gc.y * c1 + 2.f * Gv.y * v1) / W1;
        const float a30 = 2.f * Gv.x / (W0 * W0), a31 = 2.f * Gv.y / (W1 * W1);
        // pass 2: gradient of the loss with respect to each weight
        float self0 = 0.f, self1 = 0.f, Gil0 = 0.f, Gil1 = 0.f;
        for (int j = -2; j <= 2; ++j)
            for (int i = -2; i <= 2; ++i) {
                if (!i && !j) continue;
                const int qx = px + i * step, qy = py + j * step;
                if (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H) continue;
                const int q = qy * k.W + qx;
                const float4 cq = __ldg(x + q);
                if (!fg_var(cq.z)) continue;
                const TapW t = tap_weight<kNsq>(k, step, i, j, zp, gz, cp.x, cp.y, il0, il1, S::g(g, q), cq.x, cq.y);
                const float Gw0 = a10 * cq.x - a20 + a30 * t.w0 * cq.z;
                const float Gw1 = a11 * cq.y - a21 + a31 * t.w1 * cq.w;
                const float d0 = cp.x - cq.x, d1 = cp.y - cq.y;
                if (k.wl_in_atrous) {
                    self0 -= Gw0 * t.w0 * il0 * sgnf(d0);
                    self1 -= Gw1 * t.w1 * il1 * sgnf(d1);
                    Gil0 -= Gw0 * t.w0 * fabsf(d0);
                    Gil1 -= Gw1 * t.w1 * fabsf(d1);
                }
                const float gw01 = Gw0 * t.w0 + Gw1 * t.w1;
                gsz += gw01 * t.dz * t.a_off * rcp_approx(t.D * t.D);
                if (t.nd > 0.f) gsn += gw01 * __logf(t.nd);
            }
        float Gg0 = 0.f, Gg1 = 0.f;
        if (k.wl_in_atrous) {
            gsl += Gil0 * (-il0 * il0 * root0) + Gil1 * (-il1 * il1 * root1);
            // d sqrt(g)/dg is taken as 0 below g = 1e-12 (it grows without bound
            // toward g = 0, where the weight is already insensitive)
            if (root0 > 1e-6f) Gg0 = Gil0 * (-il0 * il0 * k.sigma_l * 0.5f / root0) / gw;
            if (root1 > 1e-6f) Gg1 = Gil1 * (-il1 * il1 * k.sigma_l * 0.5f / root1) / gw;
        }
        rec[4 * p + 0] = make_float4(a10, a20, a30, il0);
        rec[4 * p + 1] = make_float4(a11, a21, a31, il1);
        rec[4 * p + 2] = make_float4(Gg0, Gg1, self0, self1);
        rec[4 * p + 3] = make_float4(gz.x, gz.y, 0.f, 0.f);
    }
    block_sum3(gsz, gsn, gsl, partial);
}

// pass B: gradient with respect to the level's input colour and variance
template <int kNsq>
__global__ void __launch_bounds__(kThreadsA) atrous_bwd_b(SvgfConsts k, int step, const float4* g, const float4* x,
                                                          const float4* rec, float2* gc_in, float2* gv_in) {
    using S = Store<DHR_FP32>;
    const int qx = blockIdx.x * kBX + threadIdx.x, qy = blockIdx.y * kBY + threadIdx.y;
    if (qx >= k.W || qy >= k.H) return;
    const int q = qy * k.W + qx;
    const float4 cq = __ldg(x + q);
    if (!fg_var(cq.z)) {
        gc_in[q] = make_float2(0.f, 0.f);
        gv_in[q] = make_float2(0.f, 0.f);
        return;
    }
    const float4 zq = S::g(g, q);
    const float kc = 0.375f * 0.375f;
    const float4 r0 = rec[4 * q + 0], r1 = rec[4 * q + 1], r2 = rec[4 * q + 2];
    // own colour through the weights of q's own footprint, and the centre tap
    float gcx = r2.z + r0.x * kc, gcy = r2.w + r1.x * kc;
    float gvx = 0.5f * r0.z * kc * kc, gvy = 0.5f * r1.z * kc * kc;
    // variance Gaussians that read q
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int px = qx + dx, py = qy + dy;
            if (px < 0 || py < 0 || px >= k.W || py >= k.H) continue;
            const int p = py * k.W + px;
            if (!fg_var(__ldg(x + p).z)) continue;
            const float kk = (dx == 0 ? 0.5f : 0.25f) * (dy == 0 ? 0.5f : 0.25f);
            const float4 rp = rec[4 * p + 2];
            gvx = fmaf(rp.x, kk, gvx);
            gvy = fmaf(rp.y, kk, gvy);
        }
    // footprints of the 24 pixels p = q - (i, j) step that tap q at (i, j)
    for (int j = -2; j <= 2; ++j)
        for (int i = -2; i <= 2; ++i) {
            if (!i && !j) continue;
            const int px = qx - i * step, py = qy - j * step;
            if (px < 0 || py < 0 || px >= k.W || py >= k.H) continue;
            const int p = py * k.W + px;
            const float4 cp = __ldg(x + p);
            if (!fg_var(cp.z)) continue;
            const float4 p0 = rec[4 * p + 0], p1 = rec[4 * p + 1], p3 = rec[4 * p + 3];
            const TapW t = tap_weight<kNsq>(k, step, i, j, S::g(g, p), make_float2(p3.x, p3.y), cp.x, cp.y, p0.w,
                                            p1.w, zq, cq.x, cq.y);
            const float Gw0 = p0.x * cq.x - p0.y + p0.z * t.w0 * cq.z;
            const float Gw1 = p1.x * cq.y - p1.y + p1.z * t.w1 * cq.w;
            gcx += p0.x * t.w0 + Gw0 * t.w0 * p0.w * sgnf(cp.x - cq.x);
            gcy += p1.x * t.w1 + Gw1 * t.w1 * p1.w * sgnf(cp.y - cq.y);
            gvx = fmaf(0.5f * p0.z, t.w0 * t.w0, gvx);
            gvy = fmaf(0.5f * p1.z, t.w1 * t.w1, gvy);
        }
    gc_in[q] = make_float2(gcx, gcy);
    gv_in[q] = make_float2(gvx, gvy);
}

// upstream gradient of the last level: planes [2][N] -> float2 (+ history term)
__global__ void gather_planes_kernel(int n, const float* g_out, const float2* add, float2* gc, float2* gv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float2 v = make_float2(g_out[i], g_out[n + i]);
    if (add) {
        const float2 a = add[i];
        v.x += a.x;
        v.y += a.y;
    }
    gc[i] = v;
    gv[i] = make_float2(0.f, 0.f);
}

__global__ void add2_kernel(int n, float2* a, const float2* b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 u = a[i], v = b[i];
    a[i] = make_float2(u.x + v.x, u.y + v.y);
}

// Backward of the temporal step of one frame (FP32 storage).
__global__ void __launch_bounds__(kThreadsA) temporal_bwd_kernel(
    SvgfConsts k, dhr_camera cam, dhr_camera cam_prev, const float4* g_cur, const uint32_t* mesh_cur,
    const float4* g_prev, const uint32_t* mesh_prev, const float* sig, const float4* mom, const uint8_t* hist,
    const float2* gc, const float2* gv, const float4* gmom, float* g_sig, float2* gcol_prev, float4* gmom_prev,
    float* partial) {
    using S = Store<DHR_FP32>;
    const int x = blockIdx.x * kBX + threadIdx.x, y = blockIdx.y * kBY + threadIdx.y;
    const int N = k.W * k.H;
    float gsz = 0.f, gsn = 0.f;
    const bool inside = x < k.W && y < k.H;
    const int p = inside ? y * k.W + x : 0;
    const float4 zn = inside ? S::g(g_cur, p) : make_float4(INFINITY, 0.f, 0.f, 0.f);
    if (inside && is_fg(zn.x)) {
        const int n = hist[p];
        const float2 gz = depth_grad<S>(g_cur, k.W, k.H, x, y, zn.x);
        Reproj r;
        bool valid = false;
        if (g_prev && n >= 2) {
            const float slope = fmaxf(fabsf(gz.x), fabsf(gz.y));
            valid = reproject<S>(cam, cam_prev, k.W, k.H, x, y, zn, __ldg(mesh_cur + p), slope, g_prev, mesh_prev, r);
        }
        const float a = valid ? (k.fixed_alpha ? k.alpha : fmaxf(k.alpha, 1.0f / (float)n)) : 1.0f;
        const float2 s = make_float2(sig[p], sig[N + p]);
        float2 Gce = make_float2(0.f, 0.f);
        float4 Gm = gmom[p];
        const float2 Gc = gc[p], Gv = gv[p];
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
        } else {
            // 7x7 estimate: colour = m1, var = max(0, m2 - m1^2), m_k = sum w s^k / sum w
            float sw = 0.f, s1x = 0.f, s1y = 0.f, s2x = 0.f, s2y = 0.f;
            for (int dy = -3; dy <= 3; ++dy)
                for (int dx = -3; dx <= 3; ++dx) {
                    const int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H) continue;
                    const int q = qy * k.W + qx;
                    const float4 zq = S::g(g_cur, q);
                    if (!is_fg(zq.x)) continue;
                    const float w = w_spatial(k, zn.x, make_float3(zn.y, zn.z, zn.w), gz, dx, dy, zq);
                    const float sx = sig[q], sy = sig[N + q];
                    sw += w;
                    s1x = fmaf(w, sx, s1x);
                    s1y = fmaf(w, sy, s1y);
                    s2x = fmaf(w, sx * sx, s2x);
                    s2y = fmaf(w, sy * sy, s2y);
                }
            const float m1x = s1x / sw, m1y = s1y / sw, m2x = s2x / sw, m2y = s2y / sw;
            const bool vx = m2x - m1x * m1x > 0.f, vy = m2y - m1y * m1y > 0.f;
            const float G1x = Gc.x - (vx ? 2.f * m1x * Gv.x : 0.f), G1y = Gc.y - (vy ? 2.f * m1y * Gv.y : 0.f);
            const float G2x = vx ? Gv.x : 0.f, G2y = vy ? Gv.y : 0.f;
            for (int dy = -3; dy <= 3; ++dy)
                for (int dx = -3; dx <= 3; ++dx) {
                    const int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qy < 0 || qx >= k.W || qy >= k.H) continue;
                    const int q = qy * k.W + qx;
                    const float4 zq = S::g(g_cur, q);
                    if (!is_fg(zq.x)) continue;
                    float a_off = 0.f, D = 1.f, nd = 1.f;
                    if (dx || dy) {
                        a_off = fabsf(fmaf(gz.x, (float)-dx, gz.y * (float)-dy));
                        D = fmaf(k.sigma_z, a_off, k.eps_z);
                        nd = zn.y * zq.y + zn.z * zq.z + zn.w * zq.w;
                    }
                    const float w = w_spatial(k, zn.x, make_float3(zn.y, zn.z, zn.w), gz, dx, dy, zq);
                    const float sx = sig[q], sy = sig[N + q];
                    atomicAdd(g_sig + q, (G1x + G2x * 2.f * sx) * w / sw);
                    atomicAdd(g_sig + N + q, (G1y + G2y * 2.f * sy) * w / sw);
                    if (dx || dy) {
                        const float Gw = (G1x * (sx - m1x) + G2x * (sx * sx - m2x) + G1y * (sy - m1y) +
                                          G2y * (sy * sy - m2y)) / sw;
                        gsz += Gw * w * fabsf(zn.x - zq.x) * a_off * rcp_approx(D * D);
                        if (nd > 0.f) gsn += Gw * w * __logf(nd);
                    }
                }
        }
        // moving averages
        atomicAdd(g_sig + p, a * Gce.x + a * Gm.x + 2.f * a * s.x * Gm.z);
        atomicAdd(g_sig + N + p, a * Gce.y + a * Gm.y + 2.f * a * s.y * Gm.w);
        if (valid) {
            const float b = 1.f - a;
            for (int t = 0; t < 4; ++t) {
                if (!(r.ok & (1 << t))) continue;
                const int q = (r.y0 + (t >> 1)) * k.W + (r.x0 + (t & 1));
                const float beta = r.w[t] / r.sumw;
                atomicAdd(&gcol_prev[q].x, beta * b * Gce.x);
                atomicAdd(&gcol_prev[q].y, beta * b * Gce.y);
                atomicAdd(&gmom_prev[q].x, beta * b * Gm.x);
                atomicAdd(&gmom_prev[q].y, beta * b * Gm.y);
                atomicAdd(&gmom_prev[q].z, beta * b * Gm.z);
                atomicAdd(&gmom_prev[q].w, beta * b * Gm.w);
            }
        }
    }
    block_sum3(gsz, gsn, 0.f, partial);
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
    float4* illum = nullptr;   // [F][N] temporal outputs
    float4* mom = nullptr;     // [F][N] moments
    uint8_t* hist = nullptr;   // [F][N] history lengths
    float2* col = nullptr;     // [N] colour history (forward)
    float4* lev[2] = {nullptr, nullptr};
    float4* lvin = nullptr;    // [levels - 1][N] inputs of levels 1.. (backward scratch)
    int lvin_levels = 0;
    float2* gc[2] = {nullptr, nullptr};
    float2* gv[2] = {nullptr, nullptr};
    float2* gcol[2] = {nullptr, nullptr};
    float4* gmom[2] = {nullptr, nullptr};
    float4* rec = nullptr;     // [N][4]
    float* partial = nullptr;  // [blocks][3]
    double* acc = nullptr;     // [3]
    int nblocks = 0;
};

using namespace dhr;

static void tape_free(dhr_svgf_tape* t) {
    if (!t) return;
    cudaFree(t->illum);
    cudaFree(t->mom);
    cudaFree(t->hist);
    cudaFree(t->col);
    for (int i = 0; i < 2; ++i) {
        cudaFree(t->lev[i]);
        cudaFree(t->gc[i]);
        cudaFree(t->gv[i]);
        cudaFree(t->gcol[i]);
        cudaFree(t->gmom[i]);
    }
    cudaFree(t->rec);
    cudaFree(t->lvin);
    cudaFree(t->partial);
    cudaFree(t->acc);
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
        if (!e) e = cudaMalloc((void**)&t->gc[i], n * 8);
        if (!e) e = cudaMalloc((void**)&t->gv[i], n * 8);
        if (!e) e = cudaMalloc((void**)&t->gcol[i], n * 8);
        if (!e) e = cudaMalloc((void**)&t->gmom[i], n * 16);
    }
    if (!e) e = cudaMalloc((void**)&t->rec, n * 64);
    if (!e) e = cudaMalloc((void**)&t->partial, (size_t)t->nblocks * 3 * sizeof(float));
    if (!e) e = cudaMalloc((void**)&t->acc, 3 * sizeof(double));
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
        const float4* in = illum;
        for (int l = 0; l < L; ++l) {
            float4* o = t->lev[l & 1];
            const int mode = (l == L - 1 && L > 1) ? 2 : (l == 0 ? 1 : 0);
            DHR_TRY(launch_atrous<DHR_FP32>(mode, nsq, 2, st, k, 1 << l, gc, in, o, t->col, ao, sh));
            if (L == 1) {
                passthrough_kernel<DHR_FP32><<<(int)((N + 255) / 256), 256, 0, st>>>((int)N, o, t->col, ao, sh);
                DHR_CUDA_TRY(cudaGetLastError());
            }
            in = o;
        }
    }
    t->frames_recorded = t->F;
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
    cudaStream_t st = as_stream(stream);
    using S = Store<DHR_FP32>;
    const SvgfConsts k = make_consts(t->W, t->H, params);
    const int nsq = atrous_nsq(params);
    const size_t N = (size_t)t->W * t->H;
    const int n = (int)N;
    const dim3 blk(32, 8), grid((t->W + 31) / 32, (t->H + 7) / 8);
    const int eb = (n + 255) / 256;
    const int L = (int)params->levels;
    if (L > 1 && t->lvin_levels < L - 1) {   // inputs of levels 1..L-1, allocated on first use
        cudaFree(t->lvin);
        t->lvin = nullptr;
        t->lvin_levels = 0;
        const cudaError_t e = cudaMalloc((void**)&t->lvin, (size_t)(L - 1) * N * 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(e == cudaErrorMemoryAllocation ? DHR_ERR_OOM : DHR_ERR_CUDA,
                             "svgf_seq_backward: level scratch: %s", cudaGetErrorString(e));
        }
        t->lvin_levels = L - 1;
    }
    DHR_CUDA_TRY(cudaMemsetAsync(g_sig, 0, (size_t)t->F * 2 * N * sizeof(float), st));
    DHR_CUDA_TRY(cudaMemsetAsync(t->acc, 0, 3 * sizeof(double), st));
    DHR_CUDA_TRY(cudaMemsetAsync(t->gcol[0], 0, N * 8, st));
    DHR_CUDA_TRY(cudaMemsetAsync(t->gmom[0], 0, N * 16, st));
    int nx = 0;   // index of the "from the next frame" gradient buffers
    for (int f = t->F - 1; f >= 0; --f) {
        const auto* gcur = static_cast<const S::G*>(gbufs[f].depth_normal);
        const float4* illum = t->illum + (size_t)f * N;
        int cur = 0;
        gather_planes_kernel<<<eb, 256, 0, st>>>(n, g_out + (size_t)f * 2 * N, L == 0 ? t->gcol[nx] : nullptr,
                                                t->gc[0], t->gv[0]);
        DHR_CUDA_TRY(cudaGetLastError());
        // recompute the inputs of levels 1..L-1 from the recorded temporal output
        for (int i = 0; i + 1 < L; ++i)
            DHR_TRY(launch_atrous<DHR_FP32>(0, nsq, 2, st, k, 1 << i, gcur, i == 0 ? illum : t->lvin + (size_t)(i - 1) * N,
                                            t->lvin + (size_t)i * N, nullptr, nullptr, nullptr));
        for (int l = L - 1; l >= 0; --l) {
            const float4* xin = l == 0 ? illum : t->lvin + (size_t)(l - 1) * N;
            if (l == 0) {   // level-0 colour is also next frame's colour history
                add2_kernel<<<eb, 256, 0, st>>>(n, t->gc[cur], t->gcol[nx]);
                DHR_CUDA_TRY(cudaGetLastError());
            }
            if (nsq == 7)
                atrous_bwd_a<7><<<grid, blk, 0, st>>>(k, 1 << l, gcur, xin, t->gc[cur], t->gv[cur], t->rec, t->partial);
            else
                atrous_bwd_a<-1><<<grid, blk, 0, st>>>(k, 1 << l, gcur, xin, t->gc[cur], t->gv[cur], t->rec,
                                                       t->partial);
            DHR_CUDA_TRY(cudaGetLastError());
            reduce_partials_kernel<<<1, kReduceThreads, 0, st>>>(t->nblocks, t->partial, t->acc);
            if (nsq == 7)
                atrous_bwd_b<7><<<grid, blk, 0, st>>>(k, 1 << l, gcur, xin, t->rec, t->gc[cur ^ 1], t->gv[cur ^ 1]);
            else
                atrous_bwd_b<-1><<<grid, blk, 0, st>>>(k, 1 << l, gcur, xin, t->rec, t->gc[cur ^ 1], t->gv[cur ^ 1]);
            DHR_CUDA_TRY(cudaGetLastError());
            cur ^= 1;
        }
        const int pv = nx ^ 1;
        DHR_CUDA_TRY(cudaMemsetAsync(t->gcol[pv], 0, N * 8, st));
        DHR_CUDA_TRY(cudaMemsetAsync(t->gmom[pv], 0, N * 16, st));
        const bool hp = f > 0;
        temporal_bwd_kernel<<<grid, blk, 0, st>>>(
            k, cams[f], hp ? cams[f - 1] : cams[f], gcur, gbufs[f].mesh_id,
            hp ? static_cast<const S::G*>(gbufs[f - 1].depth_normal) : nullptr, hp ? gbufs[f - 1].mesh_id : nullptr,
            sig + (size_t)f * 2 * N, t->mom + (size_t)f * N, t->hist + (size_t)f * N, t->gc[cur], t->gv[cur],
            t->gmom[nx], g_sig + (size_t)f * 2 * N, t->gcol[pv], t->gmom[pv], t->partial);
        DHR_CUDA_TRY(cudaGetLastError());
        reduce_partials_kernel<<<1, kReduceThreads, 0, st>>>(t->nblocks, t->partial, t->acc);
        nx = pv;
    }
    finish_sigma_kernel<<<1, 32, 0, st>>>(t->acc, g_sigma);
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}
