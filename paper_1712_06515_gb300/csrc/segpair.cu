// Two-pass search: the resampling kernel writes the weighted source-frame series a_r, b_r
// of a template batch to HBM, then segpair_kernel forms every segment's spectrum on chip
// (one coset and one weight per CTA) and folds it straight into the pair sum.
//
// Compared with the one-pass cluster kernel this needs no thread-block cluster (whose
// 8-CTA placement leaves 32 of the 152 SMs idle), no distributed shared-memory gathers
// and no cluster barrier per segment; the price is one write and one read of a_r, b_r
// per template (about 0.1 ms of HBM time at the 120-day workload), with the eight coset
// CTAs of a segment reading the same rows back-to-back from L2.
//
// Pair sum (Sec. III B 1, Eq. final-formatted-rho) as in the cluster kernel's register
// form: with S = F_0 + F_1 this segment's detector sum and P the previous segment's
// (R = 1), the weight-w term of a bin is Re(conj(S) P) + Re(conj(F_1) F_0) for the
// unordered pair set, 2 Re(conj(S) P) + |S|^2 with auto-correlation included.
#include <algorithm>

#include "segpair.cuh"

namespace cc {

cc_status launch_resample(cc_plan* plan, const cc_template* t_dev, int64_t n_t, void* ab, float* norm,
                          cudaStream_t st, const KnotRec* kn = nullptr, int64_t nkn = 0, int write_inactive = 0);
cc_status launch_norm(cc_plan* plan, const float* norm, int64_t n_t, double* Dws, cudaStream_t st);
cc_status launch_knots(cc_plan* plan, const cc_template* t_dev, int64_t n_t, KnotRec* kn, cudaStream_t st);
cc_status launch_pair_finalize(cc_plan* plan, const float* raw, const double* Dws, int n_rows, int64_t n_t,
                               float* rho, cudaStream_t st);

constexpr int SP_THREADS = 256;
constexpr size_t TWO_PASS_WS_BUDGET = (size_t)24 << 30;   // a_r, b_r of one template batch



// grid: x = coset c, y = weight w * n_chunks + chunk, z = template within the batch.
// ab: [n_t][Q][2][N_tau] complex64 (bf16 pairs with BF16 storage), norm: [n_t][Q][M] (hat-A, hat-B, hat-C, 0),
// raw: [n_t][2 * n_chunks][N_f] partial pair sums.
template <int LT, bool BF16>
__global__ void __launch_bounds__(SP_THREADS, 2)
segpair_kernel(DevParams p, SegPairLayout lay, const void* __restrict__ ab, const float4* __restrict__ norm,
               float* __restrict__ raw) {
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr int L = LT;
    constexpr int PL = padded_len(L);
    constexpr int B1 = L / 16;                  // butterflies of the first (radix-16) pass
    constexpr int RLAST = last_radix(L);
    constexpr int NSL = L / RLAST;              // threads holding outputs after the last pass
    constexpr int SLP = RLAST / 2 > 0 ? RLAST / 2 : 1;   // outputs per thread with m < L/2
    constexpr bool KEEP_READS_A = pp_intermediate_passes(L) % 2 == 0;
    static_assert(B1 <= SP_THREADS && NSL <= SP_THREADS, "one butterfly per thread per pass");

    const int c = blockIdx.x;
    const int w = blockIdx.y / lay.n_chunks, chunk = blockIdx.y % lay.n_chunks;
    const int64_t t = blockIdx.z;
    const int tid = threadIdx.x, Q = p.Q;
    const int64_t N_s = p.N_s, R = p.R, M = p.M, N_tau = p.N_tau;
    const int64_t Ka = (int64_t)chunk * lay.chunk_len;
    const int64_t Kb = imin64(M, Ka + lay.chunk_len);
    const int64_t Kl = imax64(0, Ka - R);

    float2* A = (float2*)(sm + lay.off_fft);
    float2* Bf = A + PL;
    float2* H = (float2*)(sm + lay.off_h);
    const int o = __ldg(p.coset_off + c), nbc = __ldg(p.coset_off + c + 1) - o;

    float accP[SLP], cmpP[SLP];
    float2 prevP[SLP];
#pragma unroll
    for (int r = 0; r < SLP; ++r) {
        accP[r] = cmpP[r] = 0.f;
        prevP[r] = make_float2(0.f, 0.f);
    }
    const uint64_t N = (uint64_t)p.N_FFT, mask = N - 1;
    const uint64_t bc = ((uint64_t)p.b0 + (uint64_t)c) & mask;
    const float2* __restrict__ twr = p.twc + (size_t)c * N_s;
    const float4* __restrict__ nt = norm + (size_t)t * Q * M;
    const size_t abt = (size_t)t * Q * 2 * N_tau;   // element offset of this template's rows
    auto load_ab = [&](size_t i) -> float2 {
        if constexpr (BF16) return __bfloat1622float2(((const __nv_bfloat162*)ab)[i]);
        else return __ldg((const float2*)ab + i);
    };
    auto sync = []() { __syncthreads(); };

    // segment of detector X, weight w: sample r - seg0 goes to position (r - seg0 + seg0) mod L
    // (absolute r: the segment-start phase is part of the transform) times the coset
    // twiddle; first radix-16 pass in registers, stored to buf
    auto first_pass = [&](int X, int64_t seg0, float2* buf) {
        const size_t row = abt + ((size_t)X * 2 + w) * N_tau + seg0;
        const int offn = (int)((-seg0) & (int64_t)(L - 1));
        if (tid < B1) {
            float2 v[16];
            if (N_s <= L) {
                float2 vv[16], tw[16];
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int rr = (tid + r * B1 + offn) & (L - 1);
                    const bool in = rr < (int)N_s;
                    vv[r] = in ? load_ab(row + rr) : make_float2(0.f, 0.f);
                    tw[r] = in ? __ldg(twr + rr) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r] = cmul(vv[r], tw[r]);
            } else {
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    float2 acc = make_float2(0.f, 0.f);
                    for (int rr = (tid + r * B1 + offn) & (L - 1); rr < (int)N_s; rr += L)
                        acc = cadd(acc, cmul(load_ab(row + rr), __ldg(twr + rr)));
                    v[r] = acc;
                }
            }
            dft16(v);
            float2* d = buf + 17 * tid;   // padi(16 tid + r) = 17 tid + r
#pragma unroll
            for (int r = 0; r < 16; ++r) d[r] = v[r];
        }
        __syncthreads();
    };

    for (int64_t K = Kl; K < Kb; ++K) {
        const int64_t seg0 = K * N_s;
        const float2 wseg = twiddle_N((bc * ((uint64_t)seg0 & mask)) & mask, N);
        // a detector with no weight in the segment (all gaps) has F = 0
        const float4 n0 = nt[K], nl = nt[(size_t)(Q - 1) * M + K];
        const bool a0 = n0.x + n0.y > 0.f, al = nl.x + nl.y > 0.f;
        float2 v[16];
        if (Q > 1 && a0) {
            first_pass(0, seg0, A);
            stockham_pp_keep_t<L, 16>(A, Bf, tid, p.twL, sync, v);
            if (tid < NSL) {
#pragma unroll
                for (int r = 0; r < SLP; ++r)
                    if (tid + NSL * r <= lay.mmax) H[r * NSL + tid] = v[r];
            }
            if constexpr (KEEP_READS_A) __syncthreads();
        }
        if (al) {
            first_pass(Q - 1, seg0, A);
            stockham_pp_keep_t<L, 16>(A, Bf, tid, p.twL, sync, v);
        }
        if (tid < NSL) {
            const float2 wc = make_float2(wseg.x, -wseg.y);
            const bool acc_on = K >= Ka;
#pragma unroll
            for (int r = 0; r < SLP; ++r) {
                const int m = tid + NSL * r;
                if (m <= lay.mmax) {
                    const float2 Fl = al ? v[r] : make_float2(0.f, 0.f);
                    float2 F0 = Fl, F1 = make_float2(0.f, 0.f);
                    if (Q > 1) {
                        F0 = a0 ? H[r * NSL + tid] : make_float2(0.f, 0.f);
                        F1 = Fl;
                    }
                    const float2 S = cadd(F0, F1);
                    const float2 P = R > 0 ? cmul(prevP[r], wc) : make_float2(0.f, 0.f);
                    const float term = p.pair_mode == CC_PAIRS_ALL_ORDERED ? fmaf(2.f, redot(S, P), redot(S, S))
                                                                           : redot(S, P) + redot(F1, F0);
                    if (acc_on) kahan_add(accP[r], cmpP[r], term);
                    if (R > 0) prevP[r] = cmul(S, wseg);
                }
            }
        }
        // with no intermediate pass the register pass read buffer A, which the next
        // segment's first pass rewrites
        if constexpr (KEEP_READS_A) __syncthreads();
    }
    // partial sums of this (template, weight, chunk) row for the coset's bins
    __syncthreads();
    float* accm = (float*)A;
    if (tid < NSL) {
#pragma unroll
        for (int r = 0; r < SLP; ++r)
            if (tid + NSL * r <= lay.mmax) accm[tid + NSL * r] = accP[r];
    }
    __syncthreads();
    float* outp = raw + ((size_t)t * 2 * lay.n_chunks + (size_t)w * lay.n_chunks + chunk) * p.N_f;
    for (int i = tid; i < nbc; i += SP_THREADS) outp[__ldg(p.coset_k + o + i)] = accm[__ldg(p.coset_m + o + i)];
}

// ---------------------------------------------------------------------------
// Coset lengths L <= 2048: one transform per group of L/16 threads, G = min(4096 / L, 2 C)
// groups per CTA (256 threads when the template has at least 4096 / L (weight, coset)
// units, fewer otherwise), each group one unit of the same template and chunk (units
// u = w C + c, CTA x-index covering units x G .. x G + G - 1), so that every thread holds
// 16 values in every pass: the radix-16 passes have L/16 butterflies, and the last
// pass of radix R < 16 has 16 / R butterflies per thread.  (With one transform per CTA a
// 256-point transform would keep 16 of 256 threads busy.)  The template, chunk and
// segment are common to the CTA, so the detector-activity branches and the barriers are
// uniform.
template <int LT>
struct GroupedShape {
    static constexpr int L = LT;
    static constexpr int G = 4096 / L;               // transforms per 256-thread CTA (at most)
    static constexpr int GT = L / 16;                // threads per transform
    static constexpr int RLAST = last_radix(L);
    static constexpr int NSL = L / RLAST;            // butterflies of the last pass
    static constexpr int BPT = NSL / GT;             // of them per thread: 16 / RLAST
    static constexpr int SLP = RLAST / 2 > 0 ? RLAST / 2 : 1;   // kept outputs per butterfly (m < L/2)
    static constexpr int NINT = pp_intermediate_passes(L);      // radix-16 passes with NS = 16
    static_assert(G * GT == SP_THREADS && BPT * RLAST == 16, "16 values per thread in every pass");
};

template <int LT, bool BF16>
__global__ void __launch_bounds__(SP_THREADS, 2)
segpair_grouped_kernel(DevParams p, SegPairLayout lay, const void* __restrict__ ab,
                       const float4* __restrict__ norm, float* __restrict__ raw) {
    extern __shared__ __align__(16) unsigned char sm[];
    using S = GroupedShape<LT>;
    constexpr int L = S::L, PL = padded_len(L), GT = S::GT, RLAST = S::RLAST, NSL = S::NSL;
    constexpr int BPT = S::BPT, SLP = S::SLP;
    constexpr bool KEEP_READS_A = S::NINT == 0;   // the last pass reads the first pass's buffer

    const int tid = threadIdx.x, g = tid / GT, j = tid % GT;
    const int C = p.C;
    const int u = blockIdx.x * lay.grouped + g;   // (weight, coset) unit of this group
    const bool unit_ok = u < 2 * C;
    const int c = unit_ok ? u % C : 0, w = unit_ok ? u / C : 0;
    const int chunk = blockIdx.y;
    const int64_t t = blockIdx.z;
    const int Q = p.Q;
    const int64_t N_s = p.N_s, R = p.R, M = p.M, N_tau = p.N_tau;
    const int64_t Ka = (int64_t)chunk * lay.chunk_len;
    const int64_t Kb = imin64(M, Ka + lay.chunk_len);
    const int64_t Kl = imax64(0, Ka - R);
    const int Hs = lay.mmax + 1;

    float2* A = (float2*)(sm + lay.off_fft) + (size_t)g * 2 * PL;
    float2* Bf = A + PL;
    float2* H = (float2*)(sm + lay.off_h) + (size_t)g * Hs;

    float accP[BPT * SLP], cmpP[BPT * SLP];
    float2 prevP[BPT * SLP];
#pragma unroll
    for (int e = 0; e < BPT * SLP; ++e) {
        accP[e] = cmpP[e] = 0.f;
        prevP[e] = make_float2(0.f, 0.f);
    }
    const uint64_t N = (uint64_t)p.N_FFT, mask = N - 1;
    const uint64_t bc = ((uint64_t)p.b0 + (uint64_t)c) & mask;
    const float2* __restrict__ twr = p.twc + (size_t)c * N_s;
    const float4* __restrict__ nt = norm + (size_t)t * Q * M;
    const size_t abt = (size_t)t * Q * 2 * N_tau;
    auto load_ab = [&](size_t i) -> float2 {
        if constexpr (BF16) return __bfloat1622float2(((const __nv_bfloat162*)ab)[i]);
        else return __ldg((const float2*)ab + i);
    };

    // first radix-16 pass of detector X's segment (sample r - seg0 at position r mod L,
    // times the coset twiddle), stored to A
    auto first_pass = [&](int X, int64_t seg0) {
        const size_t row = abt + ((size_t)X * 2 + w) * N_tau + seg0;
        const int offn = (int)((-seg0) & (int64_t)(L - 1));
        float2 v[16];
        if (N_s <= L) {
            float2 vv[16], tw[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const int rr = (j + r * GT + offn) & (L - 1);
                const bool in = unit_ok && rr < (int)N_s;
                vv[r] = in ? load_ab(row + rr) : make_float2(0.f, 0.f);
                tw[r] = in ? __ldg(twr + rr) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = cmul(vv[r], tw[r]);
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                float2 acc = make_float2(0.f, 0.f);
                if (unit_ok)
                    for (int rr = (j + r * GT + offn) & (L - 1); rr < (int)N_s; rr += L)
                        acc = cadd(acc, cmul(load_ab(row + rr), __ldg(twr + rr)));
                v[r] = acc;
            }
        }
        dft16(v);
        float2* d = A + 17 * j;   // padi(16 j + r) = 17 j + r
#pragma unroll
        for (int r = 0; r < 16; ++r) d[r] = v[r];
    };
    // the passes after the first: an optional radix-16 pass (NS = 16) A -> B, then the
    // last pass of radix RLAST into registers, BPT butterflies per thread: butterfly
    // b = j + GT q leaves output r of its transform (bin m = b + NSL r) in o[q SLP + r]
    auto rest = [&](float2 (&o)[BPT * SLP]) {
        const float2* src = A;
        if constexpr (S::NINT == 1) {
            stockham_pass_oop_t<16, L, 16>(A, Bf, j, p.twL);
            __syncthreads();
            src = Bf;
        }
#pragma unroll
        for (int q = 0; q < BPT; ++q) {
            const int b = j + GT * q;
            float2 v[16];
            const float2* s = src + padi(b);
#pragma unroll
            for (int r = 0; r < RLAST; ++r) v[r] = s[r * pstride<NSL>()];
            apply_twiddles<RLAST>(v, p.twL, b, L - 1);
            dft_r<RLAST>(v);
#pragma unroll
            for (int r = 0; r < SLP; ++r) o[q * SLP + r] = v[r];
        }
    };

    for (int64_t K = Kl; K < Kb; ++K) {
        const int64_t seg0 = K * N_s;
        const float2 wseg = twiddle_N((bc * ((uint64_t)seg0 & mask)) & mask, N);
        const float4 n0 = nt[K], nl = nt[(size_t)(Q - 1) * M + K];
        const bool a0 = n0.x + n0.y > 0.f, al = nl.x + nl.y > 0.f;
        float2 o[BPT * SLP];
        if (Q > 1 && a0) {
            first_pass(0, seg0);
            __syncthreads();
            rest(o);
#pragma unroll
            for (int q = 0; q < BPT; ++q)
#pragma unroll
                for (int r = 0; r < SLP; ++r) {
                    const int m = j + GT * q + NSL * r;
                    if (m <= lay.mmax) H[m] = o[q * SLP + r];   // read back by this thread only
                }
            if constexpr (KEEP_READS_A) __syncthreads();   // detector 1's first pass rewrites A
        }
        if (al) {
            first_pass(Q - 1, seg0);
            __syncthreads();
            rest(o);
        }
        const float2 wc = make_float2(wseg.x, -wseg.y);
        const bool acc_on = K >= Ka;
#pragma unroll
        for (int q = 0; q < BPT; ++q)
#pragma unroll
            for (int r = 0; r < SLP; ++r) {
                const int e = q * SLP + r;
                const int m = j + GT * q + NSL * r;
                if (m <= lay.mmax) {
                    const float2 Fl = al ? o[e] : make_float2(0.f, 0.f);
                    float2 F0 = Fl, F1 = make_float2(0.f, 0.f);
                    if (Q > 1) {
                        F0 = a0 ? H[m] : make_float2(0.f, 0.f);
                        F1 = Fl;
                    }
                    const float2 Sv = cadd(F0, F1);
                    const float2 P = R > 0 ? cmul(prevP[e], wc) : make_float2(0.f, 0.f);
                    const float term = p.pair_mode == CC_PAIRS_ALL_ORDERED ? fmaf(2.f, redot(Sv, P), redot(Sv, Sv))
                                                                           : redot(Sv, P) + redot(F1, F0);
                    if (acc_on) kahan_add(accP[e], cmpP[e], term);
                    if (R > 0) prevP[e] = cmul(Sv, wseg);
                }
            }
        // with no intermediate pass the last pass read A, which the next segment's first
        // pass rewrites
        if constexpr (KEEP_READS_A) __syncthreads();
    }
    // partial sums of this group's (template, weight, chunk) row for its coset's bins
    __syncthreads();
    float* accm = (float*)A;
#pragma unroll
    for (int q = 0; q < BPT; ++q)
#pragma unroll
        for (int r = 0; r < SLP; ++r) {
            const int m = j + GT * q + NSL * r;
            if (m <= lay.mmax) accm[m] = accP[q * SLP + r];
        }
    __syncthreads();
    if (unit_ok) {
        const int o0 = __ldg(p.coset_off + c), nbc = __ldg(p.coset_off + c + 1) - o0;
        float* outp = raw + ((size_t)t * 2 * lay.n_chunks + (size_t)w * lay.n_chunks + chunk) * p.N_f;
        for (int i = j; i < nbc; i += GT) outp[__ldg(p.coset_k + o0 + i)] = accm[__ldg(p.coset_m + o0 + i)];
    }
}

static size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }
static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Whether the plan fits the two-pass kernel: Q <= 2, R <= 1, no cross-only pair set,
// coset length 64..4096, every bin in the lower half of its coset transform.
bool segpair_layout(const cc_plan* plan, int64_t n_t, SegPairLayout* lay) {
    const DevParams& p = plan->dp;
    if (p.Q > 2 || p.R > 1 || p.pair_mode == CC_PAIRS_CROSS_ONLY) return false;
    if (p.L < 64 || p.L > 4096 || plan->N_f < 1) return false;
    lay->mmax = (int)((plan->kbar.back() - plan->k0) / p.C);
    if (2 * lay->mmax >= p.L) return false;
    // L <= 2048: G transforms per CTA (segpair_grouped_kernel), each with its own buffers;
    // no more groups than the template has (weight, coset) units
    const int G = p.L <= 2048 ? std::min(4096 / (int)p.L, 2 * (int)p.C) : 1;
    lay->grouped = p.L <= 2048 ? G : 0;
    size_t o = 0;
    lay->off_fft = o;
    o = al16(o + (size_t)G * 2 * padded_len(p.L) * sizeof(float2));
    lay->off_h = o;
    o = al16(o + (size_t)G * (lay->mmax + 1) * sizeof(float2));
    lay->bytes = o;
    if (lay->bytes > 113 * 1024) return false;   // two CTAs per SM
    // chunks: about forty waves of two CTAs per SM (a short tail; measured on the 120-day
    // band: 10 -> 40 waves is 2.5 % faster), each chunk at least 4R + 1 segments
    const int64_t ctas = (int64_t)((2 * p.C + G - 1) / G) * n_t;
    // CTAs per SM: two of 256 threads, more when the grouped kernel's CTAs are smaller
    const int64_t per_sm = p.L <= 2048 ? std::max<int64_t>(2, 2 * (4096 / p.L) / G) : 2;
    const int64_t waves = plan->tuning.chunk_waves > 0 ? plan->tuning.chunk_waves : 40;
    const int64_t want = std::max<int64_t>(1, (waves * per_sm * 152 + ctas - 1) / std::max<int64_t>(ctas, 1));
    const int64_t maxch = std::max<int64_t>(1, p.M / (4 * p.R + 1));
    const int64_t nch = segpair_tma_supported(plan) ? segpair_tma_chunks(plan, n_t)
                                                    : std::min<int64_t>({want, maxch, 32767});
    lay->chunk_len = (p.M + nch - 1) / nch;
    lay->n_chunks = (int)((p.M + lay->chunk_len - 1) / lay->chunk_len);
    return true;
}

template <int LT, bool BF16>
static cudaError_t launch_segpair_t(dim3 grid, size_t smem, cudaStream_t st, const DevParams& p,
                                    const SegPairLayout& lay, const void* ab, const float4* norm, float* raw) {
    cudaError_t e = cudaFuncSetAttribute(segpair_kernel<LT, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    segpair_kernel<LT, BF16><<<grid, SP_THREADS, smem, st>>>(p, lay, ab, norm, raw);
    return cudaGetLastError();
}

template <int LT>
static cudaError_t launch_segpair_lt(dim3 grid, size_t smem, cudaStream_t st, const DevParams& p,
                                     const SegPairLayout& lay, const void* ab, const float4* norm, float* raw) {
    if (p.store == CC_STORE_BF16) return launch_segpair_t<LT, true>(grid, smem, st, p, lay, ab, norm, raw);
    return launch_segpair_t<LT, false>(grid, smem, st, p, lay, ab, norm, raw);
}

template <int LT>
static cudaError_t launch_grouped_lt(const DevParams& p, const SegPairLayout& lay, int64_t n_t, const void* ab,
                                     const float4* norm, float* raw, cudaStream_t st) {
    const int G = lay.grouped;
    const dim3 grid((unsigned)((2 * p.C + G - 1) / G), (unsigned)lay.n_chunks, (unsigned)n_t);
    const unsigned threads = (unsigned)(G * GroupedShape<LT>::GT);
    if (p.store == CC_STORE_BF16) {
        cudaError_t e = cudaFuncSetAttribute(segpair_grouped_kernel<LT, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.bytes);
        if (e != cudaSuccess) return e;
        segpair_grouped_kernel<LT, true><<<grid, threads, lay.bytes, st>>>(p, lay, ab, norm, raw);
    } else {
        cudaError_t e = cudaFuncSetAttribute(segpair_grouped_kernel<LT, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.bytes);
        if (e != cudaSuccess) return e;
        segpair_grouped_kernel<LT, false><<<grid, threads, lay.bytes, st>>>(p, lay, ab, norm, raw);
    }
    return cudaGetLastError();
}

static cudaError_t launch_segpair(const DevParams& p, const SegPairLayout& lay, int64_t n_t, const void* ab,
                                  const float4* norm, float* raw, cudaStream_t st) {
    if (lay.grouped) {
        switch (p.L) {
            case 64: return launch_grouped_lt<64>(p, lay, n_t, ab, norm, raw, st);
            case 128: return launch_grouped_lt<128>(p, lay, n_t, ab, norm, raw, st);
            case 256: return launch_grouped_lt<256>(p, lay, n_t, ab, norm, raw, st);
            case 512: return launch_grouped_lt<512>(p, lay, n_t, ab, norm, raw, st);
            case 1024: return launch_grouped_lt<1024>(p, lay, n_t, ab, norm, raw, st);
            case 2048: return launch_grouped_lt<2048>(p, lay, n_t, ab, norm, raw, st);
        }
        return cudaErrorInvalidValue;
    }
    const dim3 grid((unsigned)p.C, (unsigned)(2 * lay.n_chunks), (unsigned)n_t);
    switch (p.L) {
        case 4096: return launch_segpair_lt<4096>(grid, lay.bytes, st, p, lay, ab, norm, raw);
    }
    return cudaErrorInvalidValue;
}

// Template batch of the two-pass search and the workspace it needs.
static int64_t two_pass_batch_templates(const cc_plan* plan, int64_t n_t) {
    const size_t per_ab = (size_t)plan->Q * 2 * plan->N_tau * (plan->cfg.store == CC_STORE_BF16 ? 4 : 8) +
                          (segpair_tma_supported(plan) ? segpair_tma_fold_bytes(plan) : 0);
    int64_t b = plan->tuning.batch_templates > 0 ? plan->tuning.batch_templates
                                                 : (int64_t)std::max<size_t>(1, TWO_PASS_WS_BUDGET / per_ab);
    return std::max<int64_t>(1, std::min<int64_t>({b, n_t, 65535}));
}

static void two_pass_batch(const cc_plan* plan, int64_t n_t, const SegPairLayout& lay, int64_t* batch,
                           size_t* bytes) {
    const size_t per_ab = (size_t)plan->Q * 2 * plan->N_tau * (plan->cfg.store == CC_STORE_BF16 ? 4 : 8);
    const int64_t b = two_pass_batch_templates(plan, n_t);
    *batch = b;
    const size_t zb = segpair_tma_supported(plan) ? segpair_tma_fold_bytes(plan) : 0;
    *bytes = al256(per_ab * b) + al256(zb * b) + al256((size_t)plan->Q * plan->M * sizeof(float4) * b) +
             al256((size_t)b * sizeof(double)) + al256((size_t)b * 2 * lay.n_chunks * plan->N_f * sizeof(float)) +
             al256((size_t)b * plan->Q * knot_rows(plan) * sizeof(KnotRec)) + al256((size_t)plan->C * sizeof(int));
}

bool two_pass_supported(const cc_plan* plan) {
    SegPairLayout lay;
    return segpair_layout(plan, 1, &lay);
}

size_t two_pass_workspace_bytes(const cc_plan* plan, int64_t n_t) {
    SegPairLayout lay;
    if (n_t < 1 || !segpair_layout(plan, two_pass_batch_templates(plan, n_t), &lay)) return 0;
    int64_t batch;
    size_t bytes;
    two_pass_batch(plan, n_t, lay, &batch, &bytes);
    return bytes;
}

cc_status search_two_pass(cc_plan* plan, const cc_template* t_dev, int64_t n_t, float* rho, cudaStream_t st) {
    SegPairLayout lay;
    const size_t per_ab = (size_t)plan->Q * 2 * plan->N_tau * (plan->cfg.store == CC_STORE_BF16 ? 4 : 8);
    const int64_t b0 = two_pass_batch_templates(plan, n_t);
    if (!segpair_layout(plan, b0, &lay)) return fail(CC_ERR_UNSUPPORTED, "plan does not fit the two-pass kernel");
    int64_t batch;
    size_t bytes;
    two_pass_batch(plan, n_t, lay, &batch, &bytes);
    cc_status s = ensure_workspace(plan, bytes);
    if (s != CC_OK) return s;
    char* w = (char*)plan->ws;
    void* ab = w;
    w += al256(per_ab * batch);
    const bool tma = segpair_tma_supported(plan);
    void* zf = w;   // folded segments: the fold kernel's output
    w += al256((tma ? segpair_tma_fold_bytes(plan) : 0) * batch);
    float* nrm = (float*)w;
    w += al256((size_t)plan->Q * plan->M * sizeof(float4) * batch);
    double* D = (double*)w;
    w += al256((size_t)batch * sizeof(double));
    float* raw = (float*)w;
    w += al256((size_t)batch * 2 * lay.n_chunks * plan->N_f * sizeof(float));
    KnotRec* kn = (KnotRec*)w;
    w += al256((size_t)batch * plan->Q * knot_rows(plan) * sizeof(KnotRec));
    int* counters = (int*)w;   // unit counters of the persistent kernel
    const int64_t nkn = knot_rows(plan);
    const bool fold = tma && segpair_tma_folded(plan);
    const DevParams& p = plan->dp;
    for (int64_t t0 = 0; t0 < n_t; t0 += batch) {
        const int64_t nb = std::min(batch, n_t - t0);
        SegPairLayout lb;
        segpair_layout(plan, nb, &lb);   // chunking for this batch size (workspace sized for the largest)
        if (lb.n_chunks > lay.n_chunks) lb = lay;
        if ((s = launch_knots(plan, t_dev + t0, nb, kn, st)) != CC_OK) return s;
        if ((s = launch_resample(plan, t_dev + t0, nb, ab, nrm, st, kn, nkn)) != CC_OK) return s;
        if ((s = launch_norm(plan, nrm, nb, D, st)) != CC_OK) return s;
        cudaEvent_t ev0, ev1;
        timing_pair(plan, &ev0, &ev1);
        if (ev0) cudaEventRecord(ev0, st);
        if (tma) {
            if (fold) s = launch_fold(plan, nb, ab, (const float4*)nrm, zf, st);
            if (s == CC_OK) s = launch_segpair_tma(plan, lb, nb, fold ? zf : ab, (const float4*)nrm, raw, counters, st);
            if (ev1) cudaEventRecord(ev1, st);
            if (s != CC_OK) return s;
        } else {
            cudaError_t e = launch_segpair(p, lb, nb, ab, (const float4*)nrm, raw, st);
            count_launch();
            if (ev1) cudaEventRecord(ev1, st);
            if (e != cudaSuccess) return cuda_fail(e, "segpair launch");
        }
        if ((s = launch_pair_finalize(plan, raw, D, 2 * lb.n_chunks, nb, rho + t0 * plan->N_f, st)) != CC_OK)
            return s;
    }
    return CC_OK;
}

}  // namespace cc
