// Lossless packing of one frame's raw trace outputs for transport to the
// client (the paper streams compressed frames to its thin clients, whose
// size drives the client frame rate: Section 4.3.2, Section 5).
//
// The visibility bitmask (one bit per light) and the AO count are split
// into bit planes: planes 0 .. n_lights-1 are the lights' bits, the next
// ceil(log2(ao_spp + 1)) planes are the bits of the count.  Each plane is
// cut into 32x8-pixel tiles (row-major, ceil(W/32) x ceil(H/8)), and each
// (plane, tile) gets a 2-bit class: 0 = every pixel 0, 1 = every pixel
// inside the image 1, 2 = mixed.  Only mixed tiles carry their 256 bits.
//
// Stream (32-bit little-endian words):
//   [0] 0x56524844 ("DHRV"), [1] W, [2] H, [3] n_lights | ao_bits << 8,
//   [4] number of mixed (plane, tile) pairs M,
//   then ceil(P T / 16) words of classes, 16 per word, class of pair
//   k = plane * T + tile in bits 2 (k % 16) .. +1 of word k / 16,
//   then 8 words per mixed pair in increasing k: word r holds tile row r,
//   bit i = pixel (x0 + i, y0 + r) (0 outside the image).
// Size: 4 (5 + ceil(P T / 16) + 8 M) bytes.
#include <cub/device/device_scan.cuh>

#include "common.cuh"

namespace dhr {
namespace {

constexpr uint32_t kPackMagic = 0x56524844u;
constexpr int kPW = 32, kPH = 8, kHeader = 5;

inline int ao_bits(uint32_t spp) {
    int b = 0;
    while ((1u << b) <= spp) ++b;      // bits of the largest count, spp
    return b;
}

struct PackDims {
    int W, H, planes, tiles_x, tiles;
    int64_t pairs;
};

inline PackDims pack_dims(int W, int H, uint32_t n_lights, uint32_t spp) {
    PackDims d;
    d.W = W;
    d.H = H;
    d.planes = (int)n_lights + ao_bits(spp);
    d.tiles_x = (W + kPW - 1) / kPW;
    d.tiles = d.tiles_x * ((H + kPH - 1) / kPH);
    d.pairs = (int64_t)d.planes * d.tiles;
    return d;
}

// scratch layout: words [pairs][8] u32, mixed flags [pairs] int, offsets [pairs] int, cub temp
struct PackWork {
    uint32_t* words;
    int* mixed;
    int* offset;
    void* cub_tmp;
    size_t cub_bytes;
};

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

inline size_t cub_scan_bytes(int64_t n) {
    size_t b = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, b, (const int*)nullptr, (int*)nullptr, (int)n);
    return b;
}

inline size_t work_bytes(const PackDims& d) {
    return align256((size_t)d.pairs * 8 * 4) + 2 * align256((size_t)d.pairs * 4) + align256(cub_scan_bytes(d.pairs));
}

inline PackWork carve(void* work, const PackDims& d) {
    char* p = static_cast<char*>(work);
    PackWork w;
    w.words = reinterpret_cast<uint32_t*>(p);
    p += align256((size_t)d.pairs * 8 * 4);
    w.mixed = reinterpret_cast<int*>(p);
    p += align256((size_t)d.pairs * 4);
    w.offset = reinterpret_cast<int*>(p);
    p += align256((size_t)d.pairs * 4);
    w.cub_tmp = p;
    w.cub_bytes = cub_scan_bytes(d.pairs);
    return w;
}

// One block of 32x8 threads per tile: each warp is one tile row; the
// plane's bits of the row are one ballot.
__global__ void __launch_bounds__(256) pack_tiles_kernel(const uint8_t* mask, const uint8_t* ao, PackDims d,
                                                         int n_lights, PackWork w) {
    const int t = blockIdx.x;
    const int x = (t % d.tiles_x) * kPW + threadIdx.x, y = (t / d.tiles_x) * kPH + threadIdx.y;
    const bool in = x < d.W && y < d.H;
    const size_t p = in ? (size_t)y * d.W + x : 0;
    const uint32_t m = in ? __ldg(mask + p) : 0u, a = in ? __ldg(ao + p) : 0u;
    const uint32_t inside = __ballot_sync(0xffffffffu, in);
    __shared__ int s_any[2];
    for (int pl = 0; pl < d.planes; ++pl) {
        const uint32_t v = pl < n_lights ? (m >> pl) & 1u : (a >> (pl - n_lights)) & 1u;
        const uint32_t row = __ballot_sync(0xffffffffu, in && v);
        if (threadIdx.x == 0 && threadIdx.y == 0) s_any[0] = s_any[1] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            if (row) atomicOr(&s_any[0], 1);              // some pixel is 1
            if (row != inside) atomicOr(&s_any[1], 1);    // some inside pixel is 0
        }
        __syncthreads();
        const int64_t k = (int64_t)pl * d.tiles + t;
        if (threadIdx.x == 0) w.words[8 * k + threadIdx.y] = row;
        if (threadIdx.x == 0 && threadIdx.y == 0) w.mixed[k] = (s_any[0] && s_any[1]) ? 1 : (s_any[0] ? -1 : 0);
        __syncthreads();
    }
}

// class codes: mixed[k] = 1 mixed, -1 all one, 0 all zero (the scan below
// counts the mixed ones, so -1 is mapped to a separate pass first)
__global__ void pack_classes_kernel(PackDims d, int* mixed, uint32_t* out) {
    const int64_t word = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n_words = (d.pairs + 15) / 16;
    if (word >= n_words) return;
    uint32_t c = 0;
    for (int j = 0; j < 16; ++j) {
        const int64_t k = word * 16 + j;
        if (k >= d.pairs) break;
        const int v = mixed[k];
        c |= (uint32_t)(v == 1 ? 2 : (v == -1 ? 1 : 0)) << (2 * j);
    }
    out[kHeader + word] = c;
}

__global__ void pack_flags_kernel(int64_t n, int* mixed) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && mixed[k] != 1) mixed[k] = 0;
}

__global__ void pack_write_kernel(PackDims d, int n_lights, int ao_b, const uint32_t* words, const int* mixed,
                                  const int* offset, uint32_t* out) {
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x / 8) + threadIdx.x / 8;
    const int r = threadIdx.x & 7;
    const int64_t n_class = (d.pairs + 15) / 16;
    if (k == 0 && r == 0) {
        const int64_t last = d.pairs - 1;
        out[0] = kPackMagic;
        out[1] = (uint32_t)d.W;
        out[2] = (uint32_t)d.H;
        out[3] = (uint32_t)n_lights | ((uint32_t)ao_b << 8);
        out[4] = (uint32_t)(offset[last] + mixed[last]);
    }
    if (k >= d.pairs || !mixed[k]) return;
    out[kHeader + n_class + 8 * (int64_t)offset[k] + r] = words[8 * k + r];
}

}  // namespace
}  // namespace dhr

using namespace dhr;

extern "C" uint64_t dhr_visibility_pack_bound(int32_t width, int32_t height, uint32_t n_lights, uint32_t ao_spp) {
    if (width <= 0 || height <= 0 || n_lights < 1 || n_lights > DHR_MAX_LIGHTS || ao_spp < 1 || ao_spp > 255)
        return 0;
    const PackDims d = pack_dims(width, height, n_lights, ao_spp);
    return 4ull * (kHeader + (uint64_t)(d.pairs + 15) / 16 + 8ull * (uint64_t)d.pairs);
}

extern "C" uint64_t dhr_visibility_pack_work(int32_t width, int32_t height, uint32_t n_lights, uint32_t ao_spp) {
    if (dhr_visibility_pack_bound(width, height, n_lights, ao_spp) == 0) return 0;
    return work_bytes(pack_dims(width, height, n_lights, ao_spp));
}

extern "C" dhr_status dhr_visibility_pack(const uint8_t* shadow_mask, const uint8_t* ao_count, int32_t width,
                                          int32_t height, uint32_t n_lights, uint32_t ao_spp, void* work,
                                          uint32_t* out, void* stream) {
    clear_error();
    DHR_CHECK_ARG(shadow_mask && ao_count && work && out, "visibility_pack: null pointer");
    DHR_CHECK_ARG(dhr_visibility_pack_bound(width, height, n_lights, ao_spp) > 0,
                  "visibility_pack: bad size %dx%d, n_lights %u or ao_spp %u", width, height, n_lights, ao_spp);
    DHR_CHECK_ARG(((uintptr_t)work & 255) == 0, "visibility_pack: work must be 256-byte aligned");
    const PackDims d = pack_dims(width, height, n_lights, ao_spp);
    DHR_CHECK_ARG(d.pairs < (1ll << 30), "visibility_pack: image too large");
    cudaStream_t st = as_stream(stream);
    PackWork w = carve(work, d);
    pack_tiles_kernel<<<d.tiles, dim3(kPW, kPH), 0, st>>>(shadow_mask, ao_count, d, (int)n_lights, w);
    DHR_CUDA_TRY(cudaGetLastError());
    const int64_t n_class = (d.pairs + 15) / 16;
    pack_classes_kernel<<<(unsigned)((n_class + 255) / 256), 256, 0, st>>>(d, w.mixed, out);
    pack_flags_kernel<<<(unsigned)((d.pairs + 255) / 256), 256, 0, st>>>(d.pairs, w.mixed);
    DHR_CUDA_TRY(cudaGetLastError());
    DHR_CUDA_TRY(cub::DeviceScan::ExclusiveSum(w.cub_tmp, w.cub_bytes, w.mixed, w.offset, (int)d.pairs, st));
    pack_write_kernel<<<(unsigned)((d.pairs + 31) / 32), 256, 0, st>>>(d, (int)n_lights, ao_bits(ao_spp), w.words,
                                                                     w.mixed, w.offset, out);
    DHR_CUDA_TRY(cudaGetLastError());
    return DHR_OK;
}
