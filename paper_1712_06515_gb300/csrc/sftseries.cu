// Heterodyned, downsampled series from SFT bands (Appendix B): per SFT an N'-point
// inverse DFT of the band around k_h with the half-band index shift, the (-1)^j' sign and
// the SFT-start phase exp(-2 pi i f_h (t_K - T_sft/2)) that keeps the SFTs in phase.
// The input preparation of the search (once per dataset, not per template).
#include <cmath>
#include <vector>

#include "common.cuh"

namespace cc {
namespace {

constexpr int SS_THREADS = 256;

// one CTA per T_sft block: the block's SFT (or zeros for a gap) -> N' output samples
__global__ void __launch_bounds__(SS_THREADS)
sft_to_series_kernel(const float2* __restrict__ band, const int64_t* __restrict__ block_sft, int n_prime,
                     double T_sft, double f_h, const float2* __restrict__ tw, float2* __restrict__ x) {
    extern __shared__ __align__(16) float2 zb[];
    const int64_t b = blockIdx.x;
    const int64_t s = block_sft[b];
    float2* xo = x + b * (int64_t)n_prime;
    if (s < 0) {
        for (int j = threadIdx.x; j < n_prime; j += blockDim.x) xo[j] = make_float2(0.f, 0.f);
        return;
    }
    const float2* __restrict__ zs = band + s * (int64_t)n_prime;
    for (int m = threadIdx.x; m < n_prime; m += blockDim.x) zb[m] = __ldg(zs + m);
    __syncthreads();
    // SFT-start phase in FP64, reduced to cycles
    const double cyc = f_h * ((double)b * T_sft);
    const float c = (float)(cyc - floor(cyc));
    float sn, cs;
    sincospif(2.0f * c, &sn, &cs);
    const float2 rot = make_float2(cs, -sn);            // exp(-2 pi i c)
    const float scale = (float)(1.0 / T_sft);
    for (int j = threadIdx.x; j < n_prime; j += blockDim.x) {
        int idx = 0;                                     // (j m) mod N'
        float2 acc = make_float2(0.f, 0.f);
        for (int m = 0; m < n_prime; ++m) {
            const float2 w = tw[idx];                    // exp(+2 pi i idx / N')
            const float2 v = zb[m];
            acc.x = fmaf(v.x, w.x, fmaf(-v.y, w.y, acc.x));
            acc.y = fmaf(v.x, w.y, fmaf(v.y, w.x, acc.y));
            idx += j;
            idx -= idx >= n_prime ? n_prime : 0;
        }
        const float sg = (j & 1) ? -scale : scale;
        acc.x *= sg;
        acc.y *= sg;
        xo[j] = make_float2(fmaf(acc.x, rot.x, -acc.y * rot.y), fmaf(acc.x, rot.y, acc.y * rot.x));
    }
}

}  // namespace
}  // namespace cc

extern "C" cc_status crosscorr_sfts_to_series(const void* band_dev, const int64_t* block_sft_dev, int64_t n_blocks,
                                              int64_t n_prime, double T_sft, double f_h, void* x_dev,
                                              void* stream) {
    using namespace cc;
    if (n_blocks < 0 || n_prime < 1 || n_prime > 16384 || !(T_sft > 0) || !std::isfinite(T_sft) ||
        !std::isfinite(f_h))
        return fail(CC_ERR_INVALID, "n_blocks >= 0, 1 <= n_prime <= 16384, T_sft > 0, finite f_h required");
    if (n_blocks == 0) return CC_OK;
    if (!band_dev || !block_sft_dev || !x_dev) return fail(CC_ERR_INVALID, "null device pointer");
    if (n_blocks > 2147483647) return fail(CC_ERR_UNSUPPORTED, "more than 2^31 - 1 blocks");
    std::vector<float2> tw(n_prime);
    for (int64_t j = 0; j < n_prime; ++j) {
        const double a = 2.0 * M_PI * (double)j / (double)n_prime;
        tw[j] = make_float2((float)cos(a), (float)sin(a));
    }
    cudaStream_t st = (cudaStream_t)stream;
    float2* tw_dev = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&tw_dev, sizeof(float2) * n_prime, st);
    if (e != cudaSuccess) return cuda_fail(e, "sfts_to_series twiddles");
    if ((e = cudaMemcpyAsync(tw_dev, tw.data(), sizeof(float2) * n_prime, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess) {
        cudaFreeAsync(tw_dev, st);
        return cuda_fail(e, "sfts_to_series twiddles");
    }
    const size_t smem = sizeof(float2) * n_prime;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(sft_to_series_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess) {
        cudaFreeAsync(tw_dev, st);
        return cuda_fail(e, "sfts_to_series smem attribute");
    }
    sft_to_series_kernel<<<(unsigned)n_blocks, SS_THREADS, smem, st>>>((const float2*)band_dev, block_sft_dev,
                                                                     (int)n_prime, T_sft, f_h, tw_dev,
                                                                     (float2*)x_dev);
    count_launch();
    e = cudaGetLastError();
    cudaFreeAsync(tw_dev, st);   // stream-ordered: freed after the kernel
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "sft_to_series_kernel launch");
}
