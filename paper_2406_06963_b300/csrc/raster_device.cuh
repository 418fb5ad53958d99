// Rasterised primary visibility: the binning shared by the trace entry
// point (raster.cu) and the batched server (serve.cu).  Every triangle is
// binned into the 8 x 4-pixel tiles its clipped screen bounds overlap (one
// warp of the trace covers one such tile); the trace kernel's warp then tests
// its 32 pixel-centre rays against the tile's list with the same watertight
// test (hit_triangle) and the same rays (primary_dir) as the traversal,
// keeping per pixel the smallest (t, original index): the traversal's closest
// hit, bit for bit.  A tile whose list is longer than kMaxBin (far, dense
// geometry) or did not fit is traversed instead, with the same result.
//
// Each tile's list lives in the tile's own G-buffer depth storage (TileStore
// in trace_device.cuh), so the rasteriser needs no memory of its own; the
// list of big triangles (binned by whole blocks) lives in the mesh-id
// buffer.  Passes: clear the tile counts; bin (one block of kChunk threads
// per chunk of kChunk leaves, one thread per triangle, one warp for a
// triangle over more than 32 tiles; one over more than kBigTiles is listed);
// bin the listed big triangles, one block each.
#pragma once

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
    float3 pn[4];               // plane_dist's four planes as world-space normals: d_k = pn[k] . (P - eye)
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

// ---------------------------------------------------------------- binning
// A triangle over at most kLaneTiles tiles is binned by its own thread; one
// over more, up to kBigTiles, is listed and later binned by a warp; one over
// more than kBigTiles is listed in pieces of kBigPiece tiles, each binned by a
// whole block.  The lists let the triangles of a chunk near the camera, and
// the tiles of a triangle that fills the screen, spread over the whole GPU.
constexpr int kLaneTiles = 32;
constexpr int kBigTiles = 256;
constexpr int kBigPiece = 1024;   // 128 threads x kBatch atomics in flight
constexpr int kBigGrid = 148 * 4;

struct BinLayout {
    TileStore ts;        // the tiles' lists (G-buffer depth storage)
    uint32_t* big;       // [1 + 2 big_cap]: number of big pieces, then (leaf, piece) pairs
    uint32_t big_cap;
    uint32_t* med;       // [1 + med_cap]: number of medium triangles, then their leaves
    uint32_t med_cap;
    int tiles_x, n_tiles;
};

// Tiles first + step, first + 2 step, ... (below n) of a triangle whose tiles
// form ntx columns from (tx0, ty0): each takes the next slot of its tile's
// list (the returned count) and, if the list has room, stores the entry
// there; a count beyond the room makes the trace traverse that tile.  The
// slot atomics are issued kBatch at a time so that their round trips overlap.
constexpr int kBatch = 8;

__device__ __forceinline__ void bin_tiles(const BinLayout& b, int tx0, int ty0, int ntx, int first, int step, int n,
                                          uint32_t entry) {
    for (int i0 = first; i0 < n; i0 += step * kBatch) {
        int tx[kBatch], ty[kBatch];
        uint32_t slot[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = i0 + u * step;
            tx[u] = tx0 + (i < n ? i % ntx : 0);
            ty[u] = ty0 + (i < n ? i / ntx : 0);
            if (i < n) slot[u] = atomicAdd(tile_word(b.ts, tx[u], ty[u], 0), 1u);
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (i0 + u * step >= n) continue;
            if (slot[u] < (uint32_t)tile_capacity(b.ts, tx[u], ty[u]))
                *tile_word(b.ts, tx[u], ty[u], (int)slot[u] + 1) = entry;
        }
    }
}

// A chunk of kChunk leaves whose vertex box lies wholly outside one of the
// side planes (with a margin far above the rounding of plane_dist) holds
// only triangles that tri_bounds rejects as outside that plane: its block
// bins nothing.
__device__ __forceinline__ bool chunk_outside(const SceneView& sc, const RasterConsts& rc, int chunk) {
    const float4 lo = __ldg(sc.chunk_box + 2 * chunk), hi = __ldg(sc.chunk_box + 2 * chunk + 1);
    const float3 c = make_float3(0.5f * (lo.x + hi.x) - rc.eye.x, 0.5f * (lo.y + hi.y) - rc.eye.y,
                                 0.5f * (lo.z + hi.z) - rc.eye.z);
    const float3 h = make_float3(0.5f * (hi.x - lo.x), 0.5f * (hi.y - lo.y), 0.5f * (hi.z - lo.z));
    const float scale = fabsf(c.x) + fabsf(c.y) + fabsf(c.z) + h.x + h.y + h.z;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float3 n = rc.pn[k];
        // largest d_k over the box, against a margin of 1e-4 of the box's extent from the eye
        const float dmax = dot(n, c) + fabsf(n.x) * h.x + fabsf(n.y) * h.y + fabsf(n.z) * h.z;
        const float nn = fabsf(n.x) + fabsf(n.y) + fabsf(n.z);
        if (dmax < -1e-4f * nn * scale) return true;
    }
    return false;
}

// Bins the kChunk leaves of `chunk` (one block of kChunk threads; every
// thread of the block calls it).
__device__ __forceinline__ void bin_chunk(const SceneView& sc, const RasterConsts& rc, const BinLayout& b, int chunk) {
    if (chunk_outside(sc, rc, chunk)) return;   // uniform over the block
    const int leaf = chunk * kChunk + (int)threadIdx.x;
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    uint32_t entry = (uint32_t)leaf;
    if (leaf < sc.n_tris) {
        const float4* tr = sc.tris + 3 * leaf;
        const float3 v0 = f3(__ldg(tr)), v1 = f3(__ldg(tr + 1)), v2 = f3(__ldg(tr + 2));
        tri_bounds(rc, v0, v1, v2, x0, x1, y0, y1);
        if (sliver(v0, v1, v2)) entry |= kThinBit;
    }
    const bool any = x0 <= x1 && y0 <= y1;
    const int tx0 = x0 / kRasterTileW, tx1 = x1 / kRasterTileW, ty0 = y0 / kRasterTileH, ty1 = y1 / kRasterTileH;
    const int ntx = any ? tx1 - tx0 + 1 : 0, nty = any ? ty1 - ty0 + 1 : 0;
    const int nt = ntx * nty;
    if (nt > 0 && nt <= kLaneTiles) bin_tiles(b, tx0, ty0, ntx, 0, 1, nt, entry);
    // listed (on overflow bin_big marks every tile)
    if (nt > kBigTiles) {
        const uint32_t np = (uint32_t)((nt + kBigPiece - 1) / kBigPiece);
        const uint32_t slot = atomicAdd(b.big, np);
        if (slot + np <= b.big_cap)
            for (uint32_t c = 0; c < np; ++c) {
                b.big[1 + 2 * (slot + c)] = (uint32_t)leaf;
                b.big[2 + 2 * (slot + c)] = c;
            }
    } else if (nt > kLaneTiles) {
        const uint32_t slot = atomicAdd(b.med, 1u);
        if (slot < b.med_cap) b.med[1 + slot] = (uint32_t)leaf;
    }
}

// Bins tiles first, first + n, ... below `limit` of listed triangle `leaf`
// (its bounds as when it was listed).
__device__ __forceinline__ void bin_listed(const SceneView& sc, const RasterConsts& rc, const BinLayout& b,
                                           uint32_t leaf, int first, int n, int limit) {
    const float4* tr = sc.tris + 3 * (size_t)leaf;
    const float3 v0 = f3(__ldg(tr)), v1 = f3(__ldg(tr + 1)), v2 = f3(__ldg(tr + 2));
    int x0, x1, y0, y1;
    tri_bounds(rc, v0, v1, v2, x0, x1, y0, y1);
    if (x0 > x1 || y0 > y1) return;   // not for a listed triangle
    const uint32_t entry = leaf | (sliver(v0, v1, v2) ? kThinBit : 0u);
    const int tx0 = x0 / kRasterTileW, ty0 = y0 / kRasterTileH;
    const int ntx = x1 / kRasterTileW - tx0 + 1, nt = ntx * (y1 / kRasterTileH - ty0 + 1);
    bin_tiles(b, tx0, ty0, ntx, first, n, min(nt, limit), entry);
}

// The listed triangles: each piece of a big one by one block (threads
// stride over its kBigPiece tiles), each medium one by one warp; if a list
// overflowed, the bins are incomplete and every tile is marked to be
// traversed instead.  Block `blk` of `nblk` (every thread of the block calls
// it).
__device__ __forceinline__ void bin_big(const SceneView& sc, const RasterConsts& rc, const BinLayout& b, int blk,
                                        int nblk) {
    const uint32_t nb = b.big[0], nm = b.med[0];
    if (nb > b.big_cap || nm > b.med_cap) {
        for (int t = blk * (int)blockDim.x + (int)threadIdx.x; t < b.n_tiles; t += nblk * (int)blockDim.x)
            *tile_word(b.ts, t % b.tiles_x, t / b.tiles_x, 0) = 0xFFFFFFFFu;
        return;
    }
    const int lane = threadIdx.x & 31, wpb = (int)blockDim.x >> 5;
    for (uint32_t k = (uint32_t)(blk * wpb + ((int)threadIdx.x >> 5)); k < nm; k += (uint32_t)(nblk * wpb))
        bin_listed(sc, rc, b, b.med[1 + k], lane, 32, kBigTiles);
    for (uint32_t k = (uint32_t)blk; k < nb; k += (uint32_t)nblk) {
        const int piece = (int)b.big[2 + 2 * k];
        bin_listed(sc, rc, b, b.big[1 + 2 * k], piece * kBigPiece + (int)threadIdx.x, blockDim.x,
                   (piece + 1) * kBigPiece);
    }
}

// clears entry t of the tile counts (t == 0 also the lists' counts)
__device__ __forceinline__ void bin_clear(const BinLayout& b, int t) {
    if (t < b.n_tiles) *tile_word(b.ts, t % b.tiles_x, t / b.tiles_x, 0) = 0u;
    if (t == 0) {
        b.big[0] = 0u;
        b.med[0] = 0u;
    }
}


// Raster constants and tile layout of one frame (double, then rounded);
// false when the camera basis is singular, the image too small for the big
// list or too large for 32-bit tile indices: the caller then traverses.
__host__ __device__ inline bool make_raster(const dhr_camera& cam, void* depth_normal, uint32_t* mesh_id, int ew,
                                           RasterConsts& rc, BinLayout& b) {
    const double m[3][3] = {{cam.forward[0], cam.right[0], cam.up[0]},
                            {cam.forward[1], cam.right[1], cam.up[1]},
                            {cam.forward[2], cam.right[2], cam.up[2]}};
    const double det = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                       m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                       m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    if (!(fabs(det) > 1e-6) || !(cam.tan_half_fov_y > 0.0f)) return false;
    const int W = cam.width, H = cam.height;
    b.tiles_x = (W + kRasterTileW - 1) / kRasterTileW;
    const long long n_tiles = (long long)b.tiles_x * ((H + kRasterTileH - 1) / kRasterTileH);
    // the mesh-id buffer (W H words) holds the big list, then the medium list
    const unsigned long long words = (unsigned long long)W * H;
    b.big_cap = (uint32_t)(words / 16 < 65536 ? words / 16 : 65536);
    if (b.big_cap < 16 || n_tiles >= (1ll << 31)) return false;
    const unsigned long long med_words = words - 2 - 2ull * b.big_cap;
    b.med_cap = (uint32_t)(med_words < (1ull << 24) ? med_words : (1ull << 24));
    b.n_tiles = (int)n_tiles;
    double inv[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            const int r1 = (c + 1) % 3, r2 = (c + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
            inv[r][c] = (m[r1][c1] * m[r2][c2] - m[r1][c2] * m[r2][c1]) / det;
        }
    rc.cam = cam;
    rc.eye = make_float3(cam.pos[0], cam.pos[1], cam.pos[2]);
    rc.mf = make_float3((float)inv[0][0], (float)inv[0][1], (float)inv[0][2]);
    rc.mr = make_float3((float)inv[1][0], (float)inv[1][1], (float)inv[1][2]);
    rc.mu = make_float3((float)inv[2][0], (float)inv[2][1], (float)inv[2][2]);
    const double kx = (double)cam.tan_half_fov_y * ((double)W / (double)H), ky = cam.tan_half_fov_y;
    rc.kx = (float)kx;
    rc.ky = (float)ky;
    rc.inv_kx = (float)(1.0 / kx);
    rc.inv_ky = (float)(1.0 / ky);
    // pixel centres x in [-1, W] and y in [-1, H] (one pixel beyond the image), widened by 1e-3
    rc.sx_hi = (float)((1.0 + 1.0 / W) * kx * 1.001);
    rc.sx_lo = -rc.sx_hi;
    rc.sy_hi = (float)((1.0 + 1.0 / H) * ky * 1.001);
    rc.sy_lo = -rc.sy_hi;
    // d_k of plane_dist as world-space normals: a = (mf, mr, mu) . (P - eye), so
    // d_0 = (mr - sx_lo mf) . (P - eye) and so on
    const double sx_lo = rc.sx_lo, sx_hi = rc.sx_hi, sy_lo = rc.sy_lo, sy_hi = rc.sy_hi;
    double n[4][3];
    for (int c = 0; c < 3; ++c) {
        n[0][c] = inv[1][c] - sx_lo * inv[0][c];
        n[1][c] = sx_hi * inv[0][c] - inv[1][c];
        n[2][c] = inv[2][c] - sy_lo * inv[0][c];
        n[3][c] = sy_hi * inv[0][c] - inv[2][c];
    }
    for (int k = 0; k < 4; ++k) rc.pn[k] = make_float3((float)n[k][0], (float)n[k][1], (float)n[k][2]);
    b.ts = TileStore{reinterpret_cast<uint32_t*>(depth_normal), W, H, ew};
    b.big = mesh_id;
    b.med = mesh_id + 1 + 2 * b.big_cap;
    return true;
}

}  // namespace
}  // namespace dhr
