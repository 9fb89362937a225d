// Learned 8-tap interpolator: weight upload and tap tabulation.
//
// The network (u, nu_c) -> 64 -> 64 -> 8 taps (tanh between layers, BF16 weights,
// FP32 accumulation) depends on the sample only through u = t/dt' - floor(t/dt'),
// because nu_c is fixed by the plan's band.  So it is evaluated once per plan at
// LEARNED_NODES offsets and the resamplers interpolate the table linearly in u,
// instead of running ~4.7k multiply-adds per sample.
#include <cmath>

#include "common.cuh"

namespace cc {
namespace {

constexpr int kTabThreads = 128;
constexpr int kW1 = 0;                                           // [2][64]
constexpr int kB1 = kW1 + 2 * LEARNED_WIDTH;                     // [64]
constexpr int kW2 = kB1 + LEARNED_WIDTH;                         // [64][64]
constexpr int kB2 = kW2 + LEARNED_WIDTH * LEARNED_WIDTH;         // [64]
constexpr int kW3 = kB2 + LEARNED_WIDTH;                         // [64][8]
constexpr int kB3 = kW3 + LEARNED_WIDTH * LEARNED_TAPS;          // [8]
constexpr int kNW = kB3 + LEARNED_TAPS;
static_assert(kNW == CC_LEARNED_N_WEIGHTS, "weight count of the learned interpolator");

__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) {
    return __uint_as_float((uint32_t)b << 16);
}

// One thread per table node i: taps at u = i / (LEARNED_NODES - 1).
__global__ void __launch_bounds__(kTabThreads)
learned_taps_kernel(const uint16_t* __restrict__ wbits, float nu_feat, float* __restrict__ taps) {
    __shared__ float w[kNW];
    for (int i = threadIdx.x; i < kNW; i += blockDim.x) w[i] = bf16_bits_to_float(wbits[i]);
    __syncthreads();
    const int node = blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= LEARNED_NODES) return;
    const float s0 = 2.0f * ((float)node / (float)(LEARNED_NODES - 1)) - 1.0f;
    float h1[LEARNED_WIDTH];
#pragma unroll
    for (int o = 0; o < LEARNED_WIDTH; ++o)
        h1[o] = tanhf(fmaf(s0, w[kW1 + o], fmaf(nu_feat, w[kW1 + LEARNED_WIDTH + o], w[kB1 + o])));
    float c[LEARNED_TAPS];
#pragma unroll
    for (int n = 0; n < LEARNED_TAPS; ++n) c[n] = w[kB3 + n];
    for (int o = 0; o < LEARNED_WIDTH; ++o) {
        float a = w[kB2 + o];
#pragma unroll
        for (int i = 0; i < LEARNED_WIDTH; ++i) a = fmaf(h1[i], w[kW2 + i * LEARNED_WIDTH + o], a);
        const float h2 = tanhf(a);
#pragma unroll
        for (int n = 0; n < LEARNED_TAPS; ++n) c[n] = fmaf(h2, w[kW3 + o * LEARNED_TAPS + n], c[n]);
    }
#pragma unroll
    for (int n = 0; n < LEARNED_TAPS; ++n) taps[node * LEARNED_TAPS + n] = c[n];
}

}  // namespace
}  // namespace cc

extern "C" cc_status crosscorr_plan_set_learned_interp(cc_plan* plan, const cc_learned_interp* li) {
    CC_NVTX_RANGE("crosscorr_plan_set_learned_interp");
    using namespace cc;
    if (!plan || !li) return fail(CC_ERR_INVALID, "null argument to crosscorr_plan_set_learned_interp");
    if (plan->cfg.interp != CC_INTERP_LEARNED)
        return fail(CC_ERR_INVALID, "plan was not built with interp = CC_INTERP_LEARNED");
    if (!li->weights_bf16 || li->n_weights != CC_LEARNED_N_WEIGHTS)
        return fail(CC_ERR_INVALID, "learned interpolator needs 4872 BF16 weights");
    for (int i = 0; i < kNW; ++i)
        if ((li->weights_bf16[i] & 0x7F80u) == 0x7F80u)
            return fail(CC_ERR_INVALID, "learned interpolator weight " + std::to_string(i) + " is not finite");
    if (!std::isfinite(li->nu_lo) || !std::isfinite(li->nu_hi) || !(li->nu_lo < li->nu_hi))
        return fail(CC_ERR_INVALID, "nu_lo < nu_hi (finite) required");
    if (!(li->nu_c >= li->nu_lo && li->nu_c <= li->nu_hi))
        return fail(CC_ERR_UNSUPPORTED, "nu_c outside the range the interpolator was trained for");
    const float nu_feat = (float)((2.0 * li->nu_c - li->nu_lo - li->nu_hi) / (li->nu_hi - li->nu_lo));

    cudaError_t e;
    if (!plan->learned_w) {
        if ((e = cudaMalloc(&plan->learned_w, sizeof(uint16_t) * kNW)) != cudaSuccess) {
            plan->learned_w = nullptr;
            return cuda_fail(e, "cudaMalloc (learned weights)");
        }
    }
    if (!plan->learned_taps) {
        if ((e = cudaMalloc(&plan->learned_taps, sizeof(float) * LEARNED_NODES * LEARNED_TAPS)) != cudaSuccess) {
            plan->learned_taps = nullptr;
            return cuda_fail(e, "cudaMalloc (learned tap table)");
        }
    }
    if ((e = cudaMemcpy(plan->learned_w, li->weights_bf16, sizeof(uint16_t) * kNW, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return cuda_fail(e, "cudaMemcpy (learned weights)");
    plan->dp.ltaps = nullptr;   // unusable until the table is complete
    const int blocks = (LEARNED_NODES + kTabThreads - 1) / kTabThreads;
    learned_taps_kernel<<<blocks, kTabThreads>>>(plan->learned_w, nu_feat, plan->learned_taps);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "learned_taps_kernel launch");
    if ((e = cudaStreamSynchronize(0)) != cudaSuccess) return cuda_fail(e, "learned_taps_kernel");
    plan->dp.ltaps = plan->learned_taps;
    return CC_OK;
}
