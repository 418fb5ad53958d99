// Rasterised primary visibility.  The paper's clients rasterise the G-buffer
// (Section 1, Section 3.3).  Here every triangle is binned into the 8 x 4-pixel
// tiles its clipped screen bounds overlap (one warp of the trace covers one
// such tile), and the warp of a tile tests its 32 pixel-centre rays against
// the tile's list with the same watertight test (hit_triangle) and the same
// rays (primary_dir) as the traversal, keeping per pixel the smallest
// (t, original index): the traversal's closest hit, bit for bit.  A tile
// whose list is longer than kMaxBin (far, dense geometry) or did not fit is
// traversed instead, with the same result.
//
// Passes (all on the caller's stream): clear the tile counts; count (one
// thread per triangle, one warp for a triangle over more than 32 tiles, one
// block for one over more than kBigTiles); an exclusive scan of the counts;
// fill (the same split); then one thread per pixel writes the
// key (t bits << 32 | original index, ~0 for none) into the G-buffer's depth
// storage, which the trace kernel reads before it overwrites it.  Counts,
// offsets and lists live in the mesh-id buffer (the trace kernel overwrites
// it afterwards), so the rasteriser needs no memory of its own.
#include <cmath>

#include "trace_device.cuh"

namespace dhr {
namespace {

constexpr float kMargin = 0.05f;  // pixels

struct RasterConsts {
    dhr_camera cam;
    float3 eye;
    float3 mf, mr, mu;          // rows of [forward | right | up]^-1: (a_f, a_r, a_u) of P - eye
    float kx, ky;               // tan(half fov) * aspect, tan(half fov)
    float inv_kx, inv_ky;
    float sx_lo, sx_hi, sy_lo, sy_hi;   // pixel-centre range widened by one pixel
};

__device__ __forceinline__ float3 cam_coords(const RasterConsts& rc, float3 p) {
    const float3 c = sub(p, rc.eye);
    return make_float3(dot(rc.mf, c), dot(rc.mr, c), dot(rc.mu, c));
}

// signed distances to the four side planes of the widened frustum (>= 0 inside)
__device__ __forceinline__ void plane_dist(const RasterConsts& rc, float3 a, float d[4]) {
    d[0] = a.y - rc.sx_lo * a.x;
    d[1] = rc.sx_hi * a.x - a.y;
    d[2] = a.z - rc.sy_lo * a.x;
    d[3] = rc.sy_hi * a.x - a.z;
}

// Accumulates the pixel coordinates of camera-space point p (a_f, a_r, a_u)
// into the box; a point at the eye (a_f <= 0 after clipping) widens it to
// the whole image.
__device__ __forceinline__ void add_point(const RasterConsts& rc, float3 p, float& xmin, float& xmax, float& ymin,
                                          float& ymax) {
    const int W = rc.cam.width, H = rc.cam.height;
    if (!(p.x > 0.0f)) {
        xmin = fminf(xmin, -1.0f);
        ymin = fminf(ymin, -1.0f);
        xmax = fmaxf(xmax, (float)W);
        ymax = fmaxf(ymax, (float)H);
        return;
    }
    // pixel coordinates of the direction (sx, sy) = (a_r, a_u) / a_f; an
    // approximate reciprocal (relative error ~1e-7, ~1e-4 pixel) is well
    // inside the box's margin
    const float ir = __fdividef(1.0f, p.x);
    const float px = (p.y * ir * rc.inv_kx + 1.0f) * (0.5f * W) - 0.5f;
    const float py = (1.0f - p.z * ir * rc.inv_ky) * (0.5f * H) - 0.5f;
    xmin = fminf(xmin, px);
    xmax = fmaxf(xmax, px);
    ymin = fminf(ymin, py);
    ymax = fmaxf(ymax, py);
}

// Sutherland-Hodgman clip of the triangle against the side planes in `planes`
// (bit k = plane k), then the box of the clipped polygon's projection.
__device__ __noinline__ void clipped_box(const RasterConsts& rc, float3 a0, float3 a1, float3 a2, unsigned planes,
                                         float& xmin, float& xmax, float& ymin, float& ymax) {
    // A convex polygon gains at most one vertex per plane (3 -> 7); rounding
    // near a frustum corner could add more, so every write is checked and an
    // overflow takes the whole image (conservative).
    constexpr int kMaxV = 12;
    float3 a[2][kMaxV];
    a[0][0] = a0;
    a[0][1] = a1;
    a[0][2] = a2;
    int n = 3, cur = 0;
    for (int k = 0; k < 4; ++k) {
        if (!((planes >> k) & 1u)) continue;
        int m = 0;
        for (int i = 0; i < n; ++i) {
            const float3 p = a[cur][i], q = a[cur][(i + 1) % n];
            float dp[4], dq[4];
            plane_dist(rc, p, dp);
            plane_dist(rc, q, dq);
            if (m + 2 > kMaxV) {
                add_point(rc, make_float3(0.f, 0.f, 0.f), xmin, xmax, ymin, ymax);
                return;
            }
            if (dp[k] >= 0.0f) a[cur ^ 1][m++] = p;
            if ((dp[k] >= 0.0f) != (dq[k] >= 0.0f)) {
                const float t = dp[k] / (dp[k] - dq[k]);
                a[cur ^ 1][m++] = make_float3(p.x + t * (q.x - p.x), p.y + t * (q.y - p.y), p.z + t * (q.z - p.z));
            }
        }
        n = m;
        cur ^= 1;
        if (n == 0) return;
    }
    for (int i = 0; i < n; ++i) add_point(rc, a[cur][i], xmin, xmax, ymin, ymax);
}

// Pixel bounds [x0, x1] x [y0, y1] of the triangle's projection, widened by
// kMargin, clamped to the image; x0 > x1 when it covers no pixel centre.
// Triangles crossing a side plane of the (widened) frustum are clipped
// against those planes first, so every projected vertex lies in front of
// the eye and inside the frustum.
__device__ __forceinline__ void tri_bounds(const RasterConsts& rc, float3 v0, float3 v1, float3 v2, int& x0, int& x1,
                                           int& y0, int& y1) {
    x0 = y0 = 0;
    x1 = y1 = -1;
    const float3 a0 = cam_coords(rc, v0), a1 = cam_coords(rc, v1), a2 = cam_coords(rc, v2);
    float d0[4], d1[4], d2[4];
    plane_dist(rc, a0, d0);
    plane_dist(rc, a1, d1);
    plane_dist(rc, a2, d2);
    unsigned out_all = 0, out_any = 0;
    for (int k = 0; k < 4; ++k) {
        const unsigned o0 = d0[k] < 0.0f, o1 = d1[k] < 0.0f, o2 = d2[k] < 0.0f;
        out_all |= (o0 & o1 & o2) << k;
        out_any |= (o0 | o1 | o2) << k;
    }
    if (out_all) return;                         // wholly outside one plane
    float xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
    if (out_any) {
        clipped_box(rc, a0, a1, a2, out_any, xmin, xmax, ymin, ymax);
    } else {
        add_point(rc, a0, xmin, xmax, ymin, ymax);
        add_point(rc, a1, xmin, xmax, ymin, ymax);
        add_point(rc, a2, xmin, xmax, ymin, ymax);
    }
    const int W = rc.cam.width, H = rc.cam.height;
    // pixel centres within kMargin of the projected box (the projection's
    // rounding is below 1e-3 pixel); clamp in float before converting
    // (NaN -> empty)
    const float fx0 = fmaxf(ceilf(xmin - kMargin), 0.0f), fx1 = fminf(floorf(xmax + kMargin), (float)(W - 1));
    const float fy0 = fmaxf(ceilf(ymin - kMargin), 0.0f), fy1 = fminf(floorf(ymax + kMargin), (float)(H - 1));
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) return;
    x0 = (int)fx0;
    x1 = (int)fx1;
    y0 = (int)fy0;
    y1 = (int)fy1;
}

// The traversal only tests a triangle whose leaf box the ray passes (slab2).
// For a triangle of (near) zero area the watertight test's edge functions are
// rounding noise and could report a hit that the box test rules out, so such
// triangles take the same box test here (scalar form of slab2's lanes, with
// tmax = +inf: the traversal's tmax is the best hit so far, and a box beyond
// it holds no hit that could win).
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

// ---------------------------------------------------------------- binning
constexpr int kTileW = 8, kTileH = 4;   // the trace's warp tile
constexpr int kMaxBin = 48;             // longer lists: traverse the tile
constexpr int kScanBlock = 1024;

constexpr int kBigTiles = 256;          // more tiles: binned by a whole block
constexpr int kBigGrid = 148 * 4;

struct BinLayout {
    uint32_t* count;     // [n_tiles]
    uint32_t* offset;    // [n_tiles + 1], exclusive scan of count
    uint32_t* bsum;      // [n_blocks] block totals of the scan
    uint32_t* big;       // [1 + big_cap]: number of big triangles, then their leaves
    uint32_t* list;      // [cap] leaf indices, tile by tile
    uint32_t n_tiles, n_blocks, big_cap, cap;
    int tiles_x;
};

// Tiles first + step, first + 2 step, ... (below n) of a triangle whose
// tiles form ntx columns from (tx0, ty0): kCount adds 1 to each tile's count
// (no value returned); else each takes a slot by atomicSub and stores the
// leaf there (dropped beyond the list's capacity: that tile is then
// traversed).  The slot atomics are issued kBatch at a time so that their
// round trips overlap.
constexpr int kBatch = 8;

// list entries: leaf index | kThinBit for a triangle of (near) zero area
constexpr uint32_t kThinBit = 0x80000000u;

template <bool kCount>
__device__ __forceinline__ void bin_tiles(const BinLayout& b, int tx0, int ty0, int ntx, int first, int step, int n,
                                          uint32_t leaf) {
    for (int i0 = first; i0 < n; i0 += step * kBatch) {
        uint32_t tile[kBatch], slot[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = i0 + u * step;
            tile[u] = i < n ? (uint32_t)((ty0 + i / ntx) * b.tiles_x + tx0 + i % ntx) : 0u;
            if (i >= n) continue;
            if (kCount) atomicAdd(b.count + tile[u], 1u);
            else slot[u] = atomicSub(b.count + tile[u], 1u);
        }
        if (kCount) continue;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (i0 + u * step >= n) continue;
            const uint32_t pos = b.offset[tile[u]] + slot[u] - 1u;
            if (pos < b.cap) b.list[pos] = leaf;
        }
    }
}

// One thread per triangle; a triangle overlapping more than 32 tiles is
// binned by its whole warp (lanes stride over its tiles), one overlapping
// more than kBigTiles is listed (count pass) for bin_big_kernel.
template <bool kCount>
__global__ void __launch_bounds__(128) bin_kernel(SceneView sc, RasterConsts rc, BinLayout b) {
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    uint32_t entry = (uint32_t)leaf;
    if (leaf < sc.n_tris) {
        const float4* tr = sc.tris + 3 * leaf;
        const float3 v0 = f3(__ldg(tr)), v1 = f3(__ldg(tr + 1)), v2 = f3(__ldg(tr + 2));
        tri_bounds(rc, v0, v1, v2, x0, x1, y0, y1);
        if (!kCount && sliver(v0, v1, v2)) entry |= kThinBit;
    }
    const bool any = x0 <= x1 && y0 <= y1;
    const int tx0 = x0 / kTileW, tx1 = x1 / kTileW, ty0 = y0 / kTileH, ty1 = y1 / kTileH;
    const int ntx = any ? tx1 - tx0 + 1 : 0, nty = any ? ty1 - ty0 + 1 : 0;
    const int nt = ntx * nty;
    if (nt > 0 && nt <= 32) bin_tiles<kCount>(b, tx0, ty0, ntx, 0, 1, nt, entry);
    if (kCount && nt > kBigTiles) {
        const uint32_t slot = atomicAdd(b.big, 1u);
        if (slot < b.big_cap) b.big[1 + slot] = (uint32_t)leaf;   // else: bins unused (all tiles traversed)
    }
    unsigned big = __ballot_sync(0xffffffffu, nt > 32 && nt <= kBigTiles);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const int s_tx0 = __shfl_sync(0xffffffffu, tx0, src), s_ty0 = __shfl_sync(0xffffffffu, ty0, src);
        const int s_ntx = __shfl_sync(0xffffffffu, ntx, src), s_nt = __shfl_sync(0xffffffffu, nt, src);
        const uint32_t s_entry = __shfl_sync(0xffffffffu, entry, src);
        bin_tiles<kCount>(b, s_tx0, s_ty0, s_ntx, lane, 32, s_nt, s_entry);
    }
}

// the listed big triangles, one block each (threads stride over its tiles)
template <bool kCount>
__global__ void __launch_bounds__(128) bin_big_kernel(SceneView sc, RasterConsts rc, BinLayout b) {
    const uint32_t n = min(b.big[0], b.big_cap);
    for (uint32_t k = blockIdx.x; k < n; k += gridDim.x) {
        const uint32_t leaf = b.big[1 + k];
        const float4* tr = sc.tris + 3 * (size_t)leaf;
        const float3 v0 = f3(__ldg(tr)), v1 = f3(__ldg(tr + 1)), v2 = f3(__ldg(tr + 2));
        int x0, x1, y0, y1;
        tri_bounds(rc, v0, v1, v2, x0, x1, y0, y1);
        const uint32_t entry = leaf | (sliver(v0, v1, v2) ? kThinBit : 0u);
        if (x0 > x1 || y0 > y1) continue;   // not for a listed triangle (same bounds as when listed)
        const int tx0 = x0 / kTileW, ty0 = y0 / kTileH;
        const int ntx = x1 / kTileW - tx0 + 1, nt = ntx * (y1 / kTileH - ty0 + 1);
        bin_tiles<kCount>(b, tx0, ty0, ntx, threadIdx.x, blockDim.x, nt, entry);
    }
}

__global__ void bin_clear_kernel(uint32_t* count, uint32_t n, uint32_t* big) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) count[i] = 0u;
    if (i == 0) big[0] = 0u;
}

// exclusive scan of count into offset, 1024 elements per block; block totals to bsum
__global__ void __launch_bounds__(kScanBlock) scan_block_kernel(const uint32_t* count, uint32_t* offset, uint32_t* bsum,
                                                                uint32_t n) {
    __shared__ uint32_t warp_tot[32];
    const uint32_t i = blockIdx.x * kScanBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t v = i < n ? count[i] : 0u;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;   // inclusive totals of warps 0..lane
    }
    __syncthreads();
    const uint32_t before = (warp ? warp_tot[warp - 1] : 0u) + x - v;
    if (i < n) offset[i] = before;
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = warp_tot[31];
}

// exclusive scan of the block totals (one block, 1024 at a time with a carry);
// offset[n] = the grand total
__global__ void __launch_bounds__(kScanBlock) scan_top_kernel(uint32_t* bsum, uint32_t nb, uint32_t* offset, uint32_t n) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += kScanBlock) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const uint32_t c = carry;
        if (i < nb) bsum[i] = c + (warp ? warp_tot[warp - 1] : 0u) + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry = c + warp_tot[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) offset[n] = carry;
}

__global__ void scan_add_kernel(uint32_t* offset, const uint32_t* bsum, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) offset[i] += bsum[i / kScanBlock];
}

// One thread per pixel, warps on the trace's 8 x 4 tiles: the closest hit of
// the pixel-centre ray among the tile's list (or by traversal), as a key.
template <bool kHalf>
__global__ void __launch_bounds__(128) primary_bin_kernel(SceneView sc, RasterConsts rc, BinLayout b,
                                                          unsigned long long* zb) {
    const int2 px = thread_pixel();
    const int W = rc.cam.width, H = rc.cam.height;
    if (px.x >= W || px.y >= H) return;
    const Ray r = make_ray(rc.eye, primary_dir(rc.cam, px.x, px.y));
    const uint32_t tile = (uint32_t)(px.y / kTileH) * b.tiles_x + (uint32_t)(px.x / kTileW);
    const uint32_t o0 = b.offset[tile], o1 = b.offset[tile + 1];
    unsigned long long key = ~0ull;
    // bins are complete unless the big-triangle list overflowed
    if (o1 - o0 <= (uint32_t)kMaxBin && o1 <= b.cap && b.big[0] <= b.big_cap) {
        float best_t = INFINITY;
        uint32_t best_o = 0xFFFFFFFFu;
        for (uint32_t j = o0; j < o1; ++j) {
            const uint32_t e = b.list[j], lf = e & ~kThinBit;
            if (lf >= (uint32_t)sc.n_tris) continue;   // only if the 32-bit offsets wrapped
            const float4* tr = sc.tris + 3 * (size_t)lf;
            const float4 p0 = __ldg(tr), p1 = __ldg(tr + 1), p2 = __ldg(tr + 2);
            const float3 v0 = f3(p0), v1 = f3(p1), v2 = f3(p2);
            if ((e & kThinBit) && !leaf_box_hit(r, v0, v1, v2)) continue;
            float t;
            float3 bc;
            if (!hit_triangle(r, v0, v1, v2, 0.0f, INFINITY, t, bc)) continue;
            const uint32_t orig = __float_as_uint(p0.w);
            if (t < best_t || (t == best_t && orig < best_o)) {
                best_t = t;
                best_o = orig;
            }
        }
        if (best_o != 0xFFFFFFFFu) key = ((unsigned long long)__float_as_uint(best_t) << 32) | best_o;
    } else {
        float tm = INFINITY;
        float3 bc;
        const int leaf = traverse<false>(sc, r, 0.0f, tm, bc);
        if (leaf >= 0) key = ((unsigned long long)__float_as_uint(tm) << 32) | __float_as_uint(__ldg(sc.tris + 3 * leaf).w);
    }
    zb[((size_t)px.y * W + px.x) * (kHalf ? 1 : 2)] = key;
}

__global__ void leaf_map_kernel(const float4* tris, int n, uint32_t* leaf_of) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    leaf_of[__float_as_uint(__ldg(tris + 3 * i).w)] = (uint32_t)i;
}

}  // namespace

dhr_status build_leaf_map(dhr_scene* sc, cudaStream_t st) {
    if (sc->n_tris == 0) return DHR_OK;
    DHR_CUDA_TRY(cudaMalloc((void**)&sc->leaf_of, (size_t)sc->n_tris * 4));
    leaf_map_kernel<<<(sc->n_tris + 255) / 256, 256, 0, st>>>(sc->tris, (int)sc->n_tris, sc->leaf_of);
    DHR_CUDA_TRY(cudaGetLastError());
    sc->bytes += (uint64_t)sc->n_tris * 4;
    return DHR_OK;
}

dhr_status launch_raster(const dhr_scene* sc, const dhr_camera* cam, dhr_gbuffer* g, cudaStream_t st,
                         bool* launched) {
    *launched = false;
    if (sc->n_tris == 0) return DHR_OK;
    // inverse of the camera basis [forward | right | up] (double, then rounded)
    const double m[3][3] = {{cam->forward[0], cam->right[0], cam->up[0]},
                            {cam->forward[1], cam->right[1], cam->up[1]},
                            {cam->forward[2], cam->right[2], cam->up[2]}};
    const double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                       m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                       m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    if (!(std::fabs(det) > 1e-6) || !(cam->tan_half_fov_y > 0.0f)) return DHR_OK;
    const int W = cam->width, H = cam->height;
    BinLayout b;
    b.tiles_x = (W + kTileW - 1) / kTileW;
    b.n_tiles = (uint32_t)b.tiles_x * (uint32_t)((H + kTileH - 1) / kTileH);
    b.n_blocks = (b.n_tiles + kScanBlock - 1) / kScanBlock;
    const uint64_t words = (uint64_t)W * H;                  // the mesh-id buffer
    b.big_cap = (uint32_t)std::min<uint64_t>(4096, std::max<uint64_t>(16, words / 64));
    const uint64_t fixed = 2ull * b.n_tiles + 1 + b.n_blocks + 1 + b.big_cap;
    if (words < fixed + 256) return DHR_OK;                  // too small: traverse
    double inv[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            const int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
            inv[r][c] = (m[r1][c1] * m[r2][c2] - m[r1][c2] * m[r2][c1]) / det;
        }
    RasterConsts rc;
    rc.cam = *cam;
    rc.eye = make_float3(cam->pos[0], cam->pos[1], cam->pos[2]);
    rc.mf = make_float3((float)inv[0][0], (float)inv[0][1], (float)inv[0][2]);
    rc.mr = make_float3((float)inv[1][0], (float)inv[1][1], (float)inv[1][2]);
    rc.mu = make_float3((float)inv[2][0], (float)inv[2][1], (float)inv[2][2]);
    const double kx = (double)cam->tan_half_fov_y * ((double)W / (double)H), ky = cam->tan_half_fov_y;
    rc.kx = (float)kx;
    rc.ky = (float)ky;
    rc.inv_kx = (float)(1.0 / kx);
    rc.inv_ky = (float)(1.0 / ky);
    // pixel centres x in [-1, W] and y in [-1, H] (one pixel beyond the image), widened by 1e-3
    rc.sx_hi = (float)((1.0 + 1.0 / W) * kx * 1.001);
    rc.sx_lo = -rc.sx_hi;
    rc.sy_hi = (float)((1.0 + 1.0 / H) * ky * 1.001);
    rc.sy_lo = -rc.sy_hi;
    uint32_t* w = g->mesh_id;
    b.count = w;
    b.offset = w + b.n_tiles;
    b.bsum = b.offset + b.n_tiles + 1;
    b.big = b.bsum + b.n_blocks;
    b.list = b.big + 1 + b.big_cap;
    b.cap = (uint32_t)std::min<uint64_t>(words - fixed, 0xFFFFFFFFull);
    const unsigned tri_blocks = (sc->n_tris + 127) / 128;
    bin_clear_kernel<<<(b.n_tiles + 255) / 256, 256, 0, st>>>(b.count, b.n_tiles, b.big);
    bin_kernel<true><<<tri_blocks, 128, 0, st>>>(sc->view(), rc, b);
    bin_big_kernel<true><<<kBigGrid, 128, 0, st>>>(sc->view(), rc, b);
    scan_block_kernel<<<b.n_blocks, kScanBlock, 0, st>>>(b.count, b.offset, b.bsum, b.n_tiles);
    scan_top_kernel<<<1, kScanBlock, 0, st>>>(b.bsum, b.n_blocks, b.offset, b.n_tiles);
    scan_add_kernel<<<(b.n_tiles + 255) / 256, 256, 0, st>>>(b.offset, b.bsum, b.n_tiles);
    bin_kernel<false><<<tri_blocks, 128, 0, st>>>(sc->view(), rc, b);
    bin_big_kernel<false><<<kBigGrid, 128, 0, st>>>(sc->view(), rc, b);
    const dim3 grid((W + 15) / 16, (H + 7) / 8);
    auto* zb = reinterpret_cast<unsigned long long*>(g->depth_normal);
    if (g->precision == DHR_FP16) primary_bin_kernel<true><<<grid, 128, 0, st>>>(sc->view(), rc, b, zb);
    else primary_bin_kernel<false><<<grid, 128, 0, st>>>(sc->view(), rc, b, zb);
    DHR_CUDA_TRY(cudaGetLastError());
    *launched = true;
    return DHR_OK;
}

}  // namespace dhr
