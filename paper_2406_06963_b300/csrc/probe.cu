// Measurement helper: the L2 read bandwidth the traversal's node and
// triangle fetches are held against (the trace kernel's data, 86 MB for the
// 776k-triangle scene, stays L2-resident across a frame).  Not a step of the
// method.
#include "common.cuh"

namespace dhr {
namespace {

// Every thread reads float4s of the buffer in a grid-stride loop, `passes`
// times over, through L2 only (ld.global.cg: no L1 allocation), and keeps a
// sum that is stored only if it equals a value the zero-filled buffer cannot
// produce, so no load can be dropped.
__global__ void __launch_bounds__(256) l2_read_kernel(const float4* __restrict__ buf, int64_t n4, int passes,
                                                      float4* sink) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int p = 0; p < passes; ++p) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    if (acc.x + acc.y + acc.z + acc.w == -1.0f) *sink = acc;
}

}  // namespace
}  // namespace dhr

extern "C" dhr_status dhr_l2_read_bandwidth(int64_t bytes, int32_t passes, float* gbs, void* stream) {
    using namespace dhr;
    clear_error();
    DHR_CHECK_ARG(gbs, "l2_read_bandwidth: null output");
    DHR_CHECK_ARG(bytes >= (1 << 20) && bytes <= (int64_t)96 << 20 && bytes % 16 == 0,
                  "l2_read_bandwidth: bytes must be a multiple of 16 in [1 MiB, 96 MiB]");
    DHR_CHECK_ARG(passes >= 1 && passes <= 1000, "l2_read_bandwidth: passes not in 1..1000");
    cudaStream_t st = as_stream(stream);
    int dev = 0, sms = 0;
    DHR_CUDA_TRY(cudaGetDevice(&dev));
    DHR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float4* buf = nullptr;
    float4* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (!e) e = cudaMalloc(&sink, sizeof(float4));
    if (!e) e = cudaMemsetAsync(buf, 0, bytes, st);
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    float best = 0.f;
    const int64_t n4 = bytes / 16;
    const int grid = sms * 8;
    if (!e) {
        l2_read_kernel<<<grid, 256, 0, st>>>(buf, n4, 1, sink);      // brings the buffer into L2
        e = cudaGetLastError();
    }
    for (int rep = 0; rep < 5 && !e; ++rep) {
        e = cudaEventRecord(e0, st);
        if (!e) {
            l2_read_kernel<<<grid, 256, 0, st>>>(buf, n4, passes, sink);
            e = cudaGetLastError();
        }
        if (!e) e = cudaEventRecord(e1, st);
        if (!e) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
        if (!e && ms > 0.f) best = fmaxf(best, (float)((double)bytes * passes / (ms * 1e-3) / 1e9));
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    if (e) return set_error(e == cudaErrorMemoryAllocation ? DHR_ERR_OOM : DHR_ERR_CUDA, "l2_read_bandwidth: %s",
                            cudaGetErrorString(e));
    *gbs = best;
    return DHR_OK;
}
