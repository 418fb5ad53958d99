// Rasterised primary visibility of the trace entry point (the paper's
// clients rasterise their G-buffer, Section 1, Section 3.3): the binning
// passes of raster_device.cuh as kernels, and the per-scene chunk boxes.
#include <cmath>

#include "raster_device.cuh"

namespace dhr {
namespace {

__global__ void __launch_bounds__(kChunk, 8) bin_kernel(SceneView sc, RasterConsts rc, BinLayout b) {
    bin_chunk(sc, rc, b, blockIdx.x);
}

__global__ void __launch_bounds__(128) bin_big_kernel(SceneView sc, RasterConsts rc, BinLayout b) {
    bin_big(sc, rc, b, blockIdx.x, gridDim.x);
}

__global__ void bin_clear_kernel(BinLayout b) { bin_clear(b, blockIdx.x * blockDim.x + threadIdx.x); }

// box of the vertices of kChunk consecutive leaves, one block per chunk
__global__ void __launch_bounds__(kChunk) chunk_box_kernel(const float4* tris, int n, float4* box) {
    const int i = blockIdx.x * kChunk + threadIdx.x;
    float3 lo = make_float3(INFINITY, INFINITY, INFINITY), hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
    if (i < n) {
        for (int v = 0; v < 3; ++v) {
            const float4 p = __ldg(tris + 3 * i + v);
            lo = make_float3(fminf(lo.x, p.x), fminf(lo.y, p.y), fminf(lo.z, p.z));
            hi = make_float3(fmaxf(hi.x, p.x), fmaxf(hi.y, p.y), fmaxf(hi.z, p.z));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
        lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
        lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
        hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
        hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
    }
    __shared__ float3 s_lo[kChunk / 32], s_hi[kChunk / 32];
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kChunk / 32; ++w) {
            lo = make_float3(fminf(lo.x, s_lo[w].x), fminf(lo.y, s_lo[w].y), fminf(lo.z, s_lo[w].z));
            hi = make_float3(fmaxf(hi.x, s_hi[w].x), fmaxf(hi.y, s_hi[w].y), fmaxf(hi.z, s_hi[w].z));
        }
        box[2 * blockIdx.x] = make_float4(lo.x, lo.y, lo.z, 0.f);
        box[2 * blockIdx.x + 1] = make_float4(hi.x, hi.y, hi.z, 0.f);
    }
}

}  // namespace

dhr_status build_chunk_boxes(dhr_scene* sc, cudaStream_t st) {
    if (sc->n_tris == 0) return DHR_OK;
    const uint32_t chunks = (sc->n_tris + kChunk - 1) / kChunk;
    DHR_CUDA_TRY(cudaMalloc((void**)&sc->chunk_box, (size_t)chunks * 32));
    chunk_box_kernel<<<chunks, kChunk, 0, st>>>(sc->tris, (int)sc->n_tris, sc->chunk_box);
    DHR_CUDA_TRY(cudaGetLastError());
    sc->bytes += (uint64_t)chunks * 32;
    return DHR_OK;
}

dhr_status launch_raster(const dhr_scene* sc, const dhr_camera* cam, dhr_gbuffer* g, cudaStream_t st,
                         bool* launched) {
    *launched = false;
    if (sc->n_tris == 0) return DHR_OK;
    RasterConsts rc;
    BinLayout b;
    if (!make_raster(*cam, g->depth_normal, g->mesh_id, g->precision == DHR_FP16 ? 2 : 4, rc, b)) return DHR_OK;
    bin_clear_kernel<<<(unsigned)((b.n_tiles + 255) / 256), 256, 0, st>>>(b);
    bin_kernel<<<(sc->n_tris + kChunk - 1) / kChunk, kChunk, 0, st>>>(sc->view(), rc, b);
    bin_big_kernel<<<kBigGrid, 128, 0, st>>>(sc->view(), rc, b);
    DHR_CUDA_TRY(cudaGetLastError());
    *launched = true;
    return DHR_OK;
}

}  // namespace dhr
