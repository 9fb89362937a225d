// Shared declarations of the two-pass search's spectrum + pair-sum kernels (segpair.cu,
// segpair_tma.cu).
#pragma once

#include "common.cuh"
#include "fft_reg.cuh"

namespace cc {

struct SegPairLayout {
    int mmax;           // largest transform position of any bin
    int n_chunks;       // segment chunks per (template, weight, coset)
    int grouped;        // L <= 2048: transforms per CTA, min(4096 / L, 2 C) (segpair_grouped_kernel)
    int pad_;
    int64_t chunk_len;  // segments per chunk
    size_t off_fft;     // [G][2][padded L] float2: out-of-place transform buffers (G = 1 for L = 4096)
    size_t off_h;       // [G][mmax + 1] float2: detector 0's kept outputs (thread-private slots)
    size_t bytes;
};

// The persistent, TMA-staged kernel for coset length 4096 (segpair_tma.cu): whether the
// plan fits it, and one launch over a template batch of the two-pass path.
bool segpair_tma_supported(const cc_plan* plan);
int segpair_tma_chunks(const cc_plan* plan, int64_t n_t);
cc_status launch_segpair_tma(cc_plan* plan, const SegPairLayout& lay, int64_t n_t, const void* ab,
                             const float4* norm, float* raw, int* counters, cudaStream_t st);
// Segments longer than the 4096-point transform: the fold kernel's output (bytes per
// template) and its launch over a template batch (z then feeds launch_segpair_tma).
bool segpair_tma_folded(const cc_plan* plan);
size_t segpair_tma_fold_bytes(const cc_plan* plan);
cc_status launch_fold(cc_plan* plan, int64_t n_t, const void* ab, const float4* norm, void* z, cudaStream_t st);
// The staged segment-FFT stage by the same kernel (spectra written instead of pair sums):
// whether the plan fits it, and one launch writing F [n_t][Q][M][2][N_f] (counters: [C4]).
bool segfft_tma_supported(const cc_plan* plan);
cc_status launch_segfft_tma(cc_plan* plan, int64_t n_t, const void* ab, float2* F, int* counters, cudaStream_t st);

}  // namespace cc
