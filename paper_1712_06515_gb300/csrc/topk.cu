// Top-k of rho over (template, bin): descending rho, ties by flat index ascending.
//
// Pass 1: each block scans a contiguous slice, keeps its best KP entries in shared
// memory and admits a new element only if it beats the current KP-th best, merging
// the admitted candidates by a bitonic sort when the candidate buffer fills.
// Pass 2: one block merges the per-block lists the same way.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace cc {

constexpr int TOPK_THREADS = 512;
constexpr int TOPK_MAX = 4096;
constexpr int TOPK_BLOCKS = 304;   // pass-1 blocks (two per SM)

// per-block lists of TOPK_MAX candidates plus the merged list, values and indices
static size_t topk_buffer_bytes() {
    return ((size_t)TOPK_BLOCKS + 1) * TOPK_MAX * (sizeof(float) + sizeof(long long)) + 64;
}

struct __align__(16) Cand {
    float v;
    int pad;
    long long idx;
};

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
    return a.v > b.v || (a.v == b.v && a.idx < b.idx);
}

// Bitonic sort of n (power of two) entries in shared memory, best first.
__device__ void bitonic_sort(Cand* s, int n) {
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
                int lo = 2 * stride * (i / stride) + (i % stride);
                int hi = lo + stride;
                bool desc_block = ((lo & size) == 0);
                Cand a = s[lo], b = s[hi];
                bool swap = desc_block ? better(b, a) : better(a, b);
                if (swap) {
                    s[lo] = b;
                    s[hi] = a;
                }
            }
        }
    }
    __syncthreads();
}

__device__ __forceinline__ Cand worst_cand() {
    Cand c;
    c.v = -INFINITY;
    c.pad = 0;
    c.idx = 0x7fffffffffffffffLL;
    return c;
}

// s holds 2*KP entries: [0, KP) the current best (sorted), [KP, 2KP) candidates.
// After the call [0, KP) holds the best KP of the union, sorted.
__device__ void merge_best(Cand* s, int KP, int ncand) {
    for (int i = KP + ncand + threadIdx.x; i < 2 * KP; i += blockDim.x) s[i] = worst_cand();
    bitonic_sort(s, 2 * KP);
}

__device__ void scan_slice(const float* __restrict__ src, const long long* __restrict__ src_idx,
                           long long begin, long long end, Cand* s, int KP, int* ncand) {
    for (int i = threadIdx.x; i < 2 * KP; i += blockDim.x) s[i] = worst_cand();
    if (threadIdx.x == 0) *ncand = 0;
    __syncthreads();
    for (long long base = begin; base < end; base += blockDim.x) {
        long long i = base + threadIdx.x;
        if (i < end) {
            Cand c;
            float v = src[i];
            c.v = isnan(v) ? -INFINITY : v;
            c.pad = 0;
            c.idx = src_idx ? src_idx[i] : i;
            if (better(c, s[KP - 1])) {
                int pos = atomicAdd(ncand, 1);
                s[KP + pos] = c;
            }
        }
        __syncthreads();
        const int n = *ncand;
        // every thread has read the count before any thread admits the next tile's
        // candidates: otherwise a fast warp's atomicAdd reaches a slow warp's read and the
        // warps disagree on whether to merge (divergent barriers, overfull buffer)
        __syncthreads();
        if (n > KP - (int)blockDim.x || base + blockDim.x >= end) {
            if (n > 0) merge_best(s, KP, n);
            if (threadIdx.x == 0) *ncand = 0;
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(TOPK_THREADS)
topk_pass1(const float* __restrict__ rho, long long n, int KP, float* out_v, long long* out_i) {
    extern __shared__ __align__(16) unsigned char smem[];
    Cand* s = (Cand*)smem;
    __shared__ int ncand;
    long long per = (n + gridDim.x - 1) / gridDim.x;
    long long b = per * blockIdx.x, e = b + per < n ? b + per : n;
    scan_slice(rho, nullptr, b, e > b ? e : b, s, KP, &ncand);
    for (int i = threadIdx.x; i < KP; i += blockDim.x) {
        out_v[(long long)blockIdx.x * KP + i] = s[i].v;
        out_i[(long long)blockIdx.x * KP + i] = s[i].idx;
    }
}

__global__ void __launch_bounds__(TOPK_THREADS)
topk_pass2(const float* __restrict__ cv, const long long* __restrict__ ci, long long n, int KP,
           float* out_v, long long* out_i) {
    extern __shared__ __align__(16) unsigned char smem[];
    Cand* s = (Cand*)smem;
    __shared__ int ncand;
    scan_slice(cv, ci, 0, n, s, KP, &ncand);
    for (int i = threadIdx.x; i < KP; i += blockDim.x) {
        out_v[i] = s[i].v;
        out_i[i] = s[i].idx;
    }
}

}  // namespace cc

extern "C" cc_status crosscorr_rho_topk(cc_plan* plan, const float* rho_dev, int64_t n_t, int k,
                                        cc_hit* hits_host, void* stream) {
    CC_NVTX_RANGE("crosscorr_rho_topk");
    using namespace cc;
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (n_t < 0 || k < 1 || k > TOPK_MAX) return fail(CC_ERR_INVALID, "need n_t >= 0 and 1 <= k <= 4096");
    if (!hits_host) return fail(CC_ERR_INVALID, "hits_host is null");
    const long long n = (long long)n_t * plan->N_f;
    if (n == 0) return CC_OK;
    if (!rho_dev) return fail(CC_ERR_INVALID, "rho_dev is null");
    cudaStream_t st = (cudaStream_t)stream;
    int KP = 1;
    while (KP < k) KP <<= 1;
    KP = std::max(KP, 2 * TOPK_THREADS);   // candidate buffer must exceed one tile
    int nb = (int)std::min<long long>(TOPK_BLOCKS, (n + 65535) / 65536);
    nb = std::max(nb, 1);
    size_t cand = (size_t)nb * KP;
    // Candidate lists live in a buffer of their own, sized once for the largest k and
    // block count, so top-k never touches (or grows) the search workspace: a search
    // queued on another stream for this plan keeps its workspace intact.
    if (!plan->topk_ws) {
        cudaError_t ea = cudaMalloc(&plan->topk_ws, topk_buffer_bytes());
        if (ea != cudaSuccess) {
            plan->topk_ws = nullptr;
            return cuda_fail(ea, "top-k candidate buffer");
        }
    }
    char* w = (char*)plan->topk_ws;
    long long* ci = (long long*)w;
    long long* fi = ci + cand;
    float* cv = (float*)(fi + KP);
    float* fv = cv + cand;
    const size_t sm = (size_t)2 * KP * sizeof(Cand);
    cudaError_t e = cudaFuncSetAttribute(topk_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(topk_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_fail(e, "topk smem attribute");
    topk_pass1<<<nb, TOPK_THREADS, sm, st>>>(rho_dev, n, KP, cv, ci);
    count_launch();
    topk_pass2<<<1, TOPK_THREADS, sm, st>>>(cv, ci, (long long)cand, KP, fv, fi);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "topk launch");
    std::vector<float> hv(KP);
    std::vector<long long> hi(KP);
    e = cudaMemcpyAsync(hv.data(), fv, sizeof(float) * KP, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hi.data(), fi, sizeof(long long) * KP, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "topk copy");
    // the stream is synchronised: report a failed bounded wait of the searches before it
    unsigned err_word = 0;
    e = cudaMemcpy(&err_word, plan->dp.err, sizeof(err_word), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    if (err_word) return crosscorr_plan_check(plan, stream);
    const int nk = (int)std::min<long long>(k, n);
    for (int i = 0; i < nk; ++i) {
        cc_hit h;
        memset(&h, 0, sizeof(h));
        h.tmpl = hi[i] / plan->N_f;
        h.bin = (int32_t)(hi[i] % plan->N_f);
        h.freq = plan->freq[h.bin];
        h.rho = hv[i];
        hits_host[i] = h;
    }
    return CC_OK;
}
