// Measured FP32 throughput of this GPU: the denominator of the spectrum kernels' roofline
// (they are bound by the plain FP32 pipes).  Every thread of a full-occupancy grid runs
// eight independent chains of fused multiply-adds; the best of three event-timed
// launches gives FMA operations x 2 flop / time.
#include "common.cuh"

namespace cc {
namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;
constexpr int PK_UNROLL = 16;

__global__ void __launch_bounds__(PK_THREADS) fp32_fma_kernel(float* out, int iters, float a) {
    float x[PK_CHAINS];
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) x[i] = threadIdx.x * 1e-3f + (float)i;
    const float b = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < PK_UNROLL; ++u)
#pragma unroll
            for (int i = 0; i < PK_CHAINS; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PK_CHAINS; ++i) s += x[i];
    if (s == 1234.5f) out[threadIdx.x] = s;   // keeps the chains live; never true for a < 1
}

}  // namespace
}  // namespace cc

extern "C" cc_status crosscorr_measure_fp32_peak(double* tflops, void* stream) {
    using namespace cc;
    if (!tflops) return fail(CC_ERR_INVALID, "tflops is null");
    *tflops = 0.0;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attributes");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp32_fma_kernel, PK_THREADS, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMallocAsync(&sink, PK_THREADS * sizeof(float), st)) != cudaSuccess) return cuda_fail(e, "sink");
    if ((e = cudaEventCreate(&e0)) == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = sms * per_sm, iters = 2048;
    double best = 0.0;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        fp32_fma_kernel<<<blocks, PK_THREADS, 0, st>>>(sink, iters, 0.999f);
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        const double flops = 2.0 * (double)blocks * PK_THREADS * iters * PK_UNROLL * PK_CHAINS;
        if (rep > 0 && ms > 0.f) best = fmax(best, flops / (ms * 1e-3) / 1e12);   // rep 0 warms up
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    if (e != cudaSuccess) return cuda_fail(e, "fp32 peak kernel");
    *tflops = best;
    return CC_OK;
}
