// Spectrum + pair-sum kernel of the two-pass search for coset length L = 4096 (the
// 120-day single band: N_FFT = 32768 = 8 cosets of 4096, N_s = 3600 samples per
// segment): a persistent kernel whose segment samples arrive by TMA bulk copies.
//
// Per (template, weight, chunk of segments, coset) unit a CTA walks the chunk's
// segments; per segment it transforms detector 0's and detector 1's samples (each the
// zero-padded N_FFT-point DFT restricted to coset c, Sec. III B 4: an L-point transform
// of the samples times exp(-2 pi i (b0 + c) s / N_FFT)) and folds the two spectra into
// the pair sum of Eq. final-formatted-rho, as segpair_kernel does.  What differs:
//
//   * staging: the N_s samples of the next (detector, segment) transform are copied
//     from HBM/L2 into shared memory by one cp.async.bulk (TMA, completion on an
//     mbarrier) issued as soon as the current transform's first pass has read the stage,
//     so the copy runs under the current transform's second and third passes instead of
//     stalling the first pass on global loads;
//   * scheduling: one CTA per SM slot (persistent), units handed out by a per-coset
//     atomic counter; a CTA starts on the coset smid mod C, so the CTAs sharing an SM
//     work on one coset and its 28.8 KB twiddle row stays in L1, and takes units of
//     other cosets once its own queue is empty (results never depend on placement);
//   * segment-relative positions: sample s of a segment sits at transform position s
//     (no wrap), so its transform T_K(m) = sum_s x_s W_N^((b0+c) s) W_L^(m s) lacks the
//     segment-start phase W_N^(k seg0_K) of bin k = b0 + c + C m.  In a pair of
//     consecutive segments that phase leaves theta(m) = W_N^(-k N_s), one constant per
//     bin: Re(conj(F_K) F_(K-1)) = Re(conj(T_K) T_(K-1) theta(m)), and the same-segment
//     terms carry no phase.  theta(m + 256) = theta(m) psi with psi = exp(2 pi i N_s / 16),
//     so each thread keeps theta of its first bin m = tid and steps by psi through its
//     eight bins m = tid + 256 r (psi = 1 when 16 divides N_s);
//   * coset twiddles without a per-sample table: the twiddle W_N^((b0+c) s) of sample
//     s = tid + 256 r splits into a factor per r (16 values per coset, applied in the first
//     pass) and a factor per thread, which passes through the first pass's DFT and is
//     absorbed into the second pass's table twiddles and the last pass's base twiddles
//     (the plan's twk table); the last pass computes only the 8 outputs m < L/2 that hold
//     output bins.
//
// The same kernel with SPECTRA set serves the staged segment-FFT stage: it writes each
// (detector, segment) transform, with its segment-start phase, to the coset's bins of F
// instead of summing pairs, and writes zeros for an all-zero staged row without
// transforming it.
//
// Waits on the mbarrier are bounded (about one second of clock): a wait that runs out
// sets bit 0 of the plan's device error word, every thread of the CTA agrees on it at
// the next barrier, the CTA waits (bounded again) for the copy still in flight and
// returns; crosscorr_plan_check reports CC_ERR_TIMEOUT.
#include <algorithm>

#include "segpair.cuh"

namespace cc {

namespace {

constexpr int TT_THREADS = 256;
constexpr int TT_L = 4096;
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;   // ~1 s at 2 GHz
constexpr int FOLD_MAX_F = 16;     // folds of a long segment onto the 4096 positions
constexpr int FOLD_MAX_C = 1024;   // cosets of a folded plan

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > WAIT_LIMIT_CYCLES) return false;
    return true;
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completing `bytes` transactions on the mbarrier.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned sm_id() {
    unsigned id;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
    return id;
}

struct TmaWork {
    int mmax;
    int n_chunks;
    int64_t chunk_len;
    int64_t units;        // (template, weight, chunk) units per coset
    uint32_t off_y, off_z, off_h, off_stage, off_bar;
    uint32_t stage_bytes;   // one staged row: N_s samples, or L folded positions
    int folded;             // N_s > L: rows of the fold kernel's output Z instead of a_r, b_r
    int n_in;               // valid positions of a staged row (N_s, or L when folded)
};

// ab: [n_t][Q][2][N_tau] complex64 (bf16 pairs with BF16 storage), or with folded
// segments (N_s > L) the fold kernel's Z [n_t][Q][2][M][C][L] in the same type; norm:
// [n_t][Q][M] (hat-A, hat-B, hat-C, 0), raw: [n_t][2 * n_chunks][N_f] partial pair
// sums, counters: [C] unit counters (zero at launch).
// SPECTRA (the staged segment-FFT stage): no pair sums; every (detector, segment)
// transform of the unit's chunk is written, with its segment-start phase W_N^(k seg0), to
// Fs[n_t][Q][M][2][N_f] at the coset's bins (norm unused: every segment is transformed).
template <bool BF16, bool SPECTRA>
__global__ void __launch_bounds__(TT_THREADS, 2)
segpair_tma_kernel(DevParams p, TmaWork q, const void* __restrict__ ab, const float4* __restrict__ norm,
                   float* __restrict__ raw, int* __restrict__ counters, float2* __restrict__ Fs) {
    extern __shared__ __align__(128) unsigned char sm[];
    constexpr int L = TT_L;
    constexpr int NSL = 256;    // butterflies of each pass = threads
    constexpr int SLP = 8;      // kept outputs per thread: m = tid + 256 r, r < 8 (m < L/2)
    float2* Y = (float2*)(sm + q.off_y);
    float2* Z = (float2*)(sm + q.off_z);
    float2* H = (float2*)(sm + q.off_h);
    unsigned char* stage = sm + q.off_stage;
    uint64_t* bar = (uint64_t*)(sm + q.off_bar);
    __shared__ int s_unit, s_coset;

    const int tid = threadIdx.x, Q = p.Q, C = p.C4;   // cosets of the 4096-point decomposition
    const int64_t N_s = p.N_s, R = p.R, M = p.M, N_tau = p.N_tau;
    const uint64_t N = (uint64_t)p.N_FFT, mask = N - 1;
    constexpr uint32_t ESZ = BF16 ? 4 : 8;

    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    bool first_unit = true;
    int my_c = (int)(sm_id() % (unsigned)C), tries = 0;   // thread 0's queue position

    for (;;) {
        if (tid == 0) {
            int u = -1;
            while (tries < C) {
                const int v = atomicAdd(counters + my_c, 1);
                if (v < q.units) {
                    u = v;
                    break;
                }
                my_c = my_c + 1 == C ? 0 : my_c + 1;   // this coset's queue is empty: help the next
                ++tries;
            }
            s_unit = u;
            s_coset = my_c;
        }
        __syncthreads();
        const int u = s_unit, c = s_coset;
        if (u < 0) break;
        const int64_t t = u / (2 * q.n_chunks);
        const int rem = u % (2 * q.n_chunks), w = rem / q.n_chunks, chunk = rem % q.n_chunks;
        const int64_t Ka = (int64_t)chunk * q.chunk_len;
        const int64_t Kb = imin64(M, Ka + q.chunk_len);
        const int64_t Kl = SPECTRA ? Ka : imax64(0, Ka - R);
        const uint64_t bc = ((uint64_t)p.b0 + (uint64_t)c) & mask;
        const float2* __restrict__ twk = p.twk + (size_t)c * 272;
        // pair phase of this thread's bins: theta = W_N^(-(bc + C tid) N_s)
        const uint64_t ct = bc + (uint64_t)C * tid;
        const float2 theta = twiddle_N((N - (ct * (uint64_t)N_s & mask)) & mask, N);
        const bool psi_one = (N_s & 15) == 0;
        float2 psi;
        sincospif(0.125f * (float)(N_s & 15), &psi.y, &psi.x);   // exp(2 pi i (N_s mod 16) / 16)
        // last pass (NS = 256): element r3 of thread tid takes W_L^(tid r3) W_N^(bc r3) =
        // W_N^(ct r3), formed from these four powers
        const float2 b1 = twiddle_N(ct & mask, N), b2 = twiddle_N((2 * ct) & mask, N);
        const float2 b4 = twiddle_N((4 * ct) & mask, N), b8 = twiddle_N((8 * ct) & mask, N);
        const float4* __restrict__ nt = SPECTRA ? nullptr : norm + (size_t)t * Q * M;
        // element offset of (template t, detector X, weight w) row
        const size_t abt = (size_t)t * Q * 2 * N_tau + (size_t)w * N_tau;
        auto active = [&](int64_t K, int X) {
            if constexpr (SPECTRA) return true;
            const float4 n = nt[(size_t)X * M + K];
            return n.x + n.y > 0.f;
        };
        // SPECTRA: the coset's bins of output row (X, K)
        const int o4 = __ldg(p.coset4_off + c), nb4 = __ldg(p.coset4_off + c + 1) - o4;
        // the transform after (K, X) in unit order (detector 0, then detector Q-1, of each
        // segment; inactive ones skipped); X = -1 starts at segment K
        auto next_after = [&](int64_t K, int X, int64_t& nK, int& nX) -> bool {
            if (X == 0 && Q > 1 && active(K, Q - 1)) {
                nK = K;
                nX = Q - 1;
                return true;
            }
            for (int64_t k = X < 0 ? K : K + 1; k < Kb; ++k) {
                if (Q > 1 && active(k, 0)) {
                    nK = k;
                    nX = 0;
                    return true;
                }
                if (active(k, Q - 1)) {
                    nK = k;
                    nX = Q - 1;
                    return true;
                }
            }
            return false;
        };
        // folded segments: the row Z_q of coset c is q = (b0 + c) mod C
        const size_t zq = (size_t)(((uint64_t)p.b0 + (uint64_t)c) & (uint64_t)(C - 1));
        auto issue = [&](int64_t K, int X) {   // thread 0, after a barrier that ends every read of the stage
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const size_t el = q.folded ? ((((size_t)t * Q + X) * 2 + w) * M + K) * C * L + zq * L
                                       : abt + (size_t)X * 2 * N_tau + (size_t)(K * N_s);
            const char* src = (const char*)ab + el * ESZ;
            mbar_arrive_expect_tx(bar, q.stage_bytes);
            tma_load_1d(stage, src, q.stage_bytes, bar);
        };

        float accP[SLP], cmpP[SLP];
        float2 prevP[SLP];
#pragma unroll
        for (int r = 0; r < SLP; ++r) {
            accP[r] = cmpP[r] = 0.f;
            prevP[r] = make_float2(0.f, 0.f);
        }
        int64_t sK = 0;   // staged transform (sK, sX)
        int sX = 0;
        bool staged = next_after(Kl, -1, sK, sX);
        // (the wait test leaves the CTA's first copy unissued: its bounded wait runs out)
        if (staged && tid == 0 && !(p.wait_test && first_unit)) issue(sK, sX);
        first_unit = false;

        for (int64_t K = Kl; K < Kb; ++K) {
            const bool a0 = active(K, 0), al = active(K, Q - 1);
            float2 v[16];
            // SPECTRA: the segment-start phase W_N^(k seg0) of bin k = bc + C m, m = tid + 256 r:
            // ph0 = W_N^((bc + C tid) seg0), stepped by W_N^(256 C seg0)
            float2 ph0 = make_float2(1.f, 0.f), phs = make_float2(1.f, 0.f);
            if constexpr (SPECTRA) {
                const uint64_t s0 = (uint64_t)(K * N_s) & mask;
                ph0 = twiddle_N(((ct & mask) * s0) & mask, N);
                phs = twiddle_N(((256 * (uint64_t)C) * s0) & mask, N);
            }
#pragma unroll 1
            for (int pass = 0; pass < 2; ++pass) {
                const int X = pass == 0 ? 0 : Q - 1;
                if (pass == 0 ? !(Q > 1 && a0) : !al) continue;   // (SPECTRA: every transform is active)
                // (K, X) is the staged transform
                const bool ok = mbar_wait(bar, phase);
                phase ^= 1;
                // first radix-16 pass: sample s = tid + 256 r of the segment (zero beyond
                // N_s) times the coset factor W_N^(256 bc r)
                bool nz = false;   // SPECTRA: a nonzero sample in this thread's share
                {
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        const int s = tid + r * 256;
                        const bool in = s < q.n_in;
                        if constexpr (BF16)
                            v[r] = in ? __bfloat1622float2(((const __nv_bfloat162*)stage)[s]) : make_float2(0.f, 0.f);
                        else
                            v[r] = in ? ((const float2*)stage)[s] : make_float2(0.f, 0.f);
                        if constexpr (SPECTRA) nz |= v[r].x != 0.f || v[r].y != 0.f;
                    }
#pragma unroll
                    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], __ldg(twk + r));
                    dft16(v);
                    float2* d = Y + 17 * tid;   // padi(16 tid + r)
#pragma unroll
                    for (int r = 0; r < 16; ++r) d[r] = v[r];
                }
                int64_t nK = 0;
                int nX = 0;
                const bool more = next_after(K, X, nK, nX);
                // every thread has read the stage and written Y; all agree on a failed wait
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) {
                        atomicOr(p.err, 1u);
                        mbar_wait(bar, phase ^ 1);   // the copy still in flight, bounded
                    }
                    __syncthreads();
                    return;
                }
                if (more && tid == 0) issue(nK, nX);
                if constexpr (SPECTRA) {
                    // a row of zeros (a gapped segment, written as zeros by the resampling
                    // stage): zero spectra, no transform
                    if (!__syncthreads_or(nz)) {
                        float2* Fo = Fs + ((((size_t)t * Q + X) * M + K) * 2 + w) * p.N_f;
                        for (int i = tid; i < nb4; i += TT_THREADS) Fo[__ldg(p.coset4_k + o4 + i)] = make_float2(0.f, 0.f);
                        continue;
                    }
                }
                // second pass (NS = 16): Y -> Z, twiddles W_L^(16 k r) W_N^(16 bc r) from the
                // table (the thread factor of the first pass's source threads)
                {
                    const int k = tid & 15;
                    const float2* s = Y + padi(tid);
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = s[r * pstride<256>()];
#pragma unroll
                    for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], __ldg(twk + 16 + r * 16 + k));
                    dft16(v);
                    float2* d = Z + padi((tid - k) * 16 + k);
#pragma unroll
                    for (int r = 0; r < 16; ++r) d[r * pstride<16>()] = v[r];
                }
                __syncthreads();
                // last pass (NS = 256) into registers: v[r] = X[tid + 256 r], r < 8
                {
                    const float2* s = Z + padi(tid);
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = s[r * pstride<256>()];
                    const float2 b3 = cmul(b2, b1);
                    v[1] = cmul(v[1], b1);
                    v[2] = cmul(v[2], b2);
                    v[3] = cmul(v[3], b3);
                    v[4] = cmul(v[4], b4);
                    v[5] = cmul(v[5], cmul(b4, b1));
                    v[6] = cmul(v[6], cmul(b4, b2));
                    v[7] = cmul(v[7], cmul(b4, b3));
                    v[8] = cmul(v[8], b8);
                    v[9] = cmul(v[9], cmul(b8, b1));
                    v[10] = cmul(v[10], cmul(b8, b2));
                    v[11] = cmul(v[11], cmul(b8, b3));
                    const float2 b12 = cmul(b8, b4);
                    v[12] = cmul(v[12], b12);
                    v[13] = cmul(v[13], cmul(b12, b1));
                    v[14] = cmul(v[14], cmul(b12, b2));
                    v[15] = cmul(v[15], cmul(b12, b3));
                    dft16_lo8(v);
                }
                if constexpr (SPECTRA) {
                    // the transform with its segment-start phase to H, then the coset's bins to F
                    float2 ph = ph0;
#pragma unroll
                    for (int r = 0; r < SLP; ++r) {
                        if (tid + NSL * r <= q.mmax) H[r * NSL + tid] = cmul(v[r], ph);
                        ph = cmul(ph, phs);
                    }
                    __syncthreads();
                    float2* Fo = Fs + ((((size_t)t * Q + X) * M + K) * 2 + w) * p.N_f;
                    for (int i = tid; i < nb4; i += TT_THREADS) Fo[__ldg(p.coset4_k + o4 + i)] = H[__ldg(p.coset4_m + o4 + i)];
                    __syncthreads();                   // H is rewritten by the next transform
                } else if (pass == 0) {
#pragma unroll
                    for (int r = 0; r < SLP; ++r)
                        if (tid + NSL * r <= q.mmax) H[r * NSL + tid] = v[r];   // read back by this thread only
                }
            }
            if constexpr (SPECTRA) continue;
            // pair terms of segment K (F = 0 for a detector with no weight in it); prevP
            // holds the previous segment's detector sum times theta of its bin
            const bool acc_on = K >= Ka;
            float2 th = theta;
#pragma unroll
            for (int r = 0; r < SLP; ++r) {
                const int m = tid + NSL * r;
                if (m <= q.mmax) {
                    const float2 Fl = al ? v[r] : make_float2(0.f, 0.f);
                    float2 F0 = Fl, F1 = make_float2(0.f, 0.f);
                    if (Q > 1) {
                        F0 = a0 ? H[r * NSL + tid] : make_float2(0.f, 0.f);
                        F1 = Fl;
                    }
                    const float2 S = cadd(F0, F1);
                    const float2 P = R > 0 ? prevP[r] : make_float2(0.f, 0.f);
                    const float term = p.pair_mode == CC_PAIRS_ALL_ORDERED ? fmaf(2.f, redot(S, P), redot(S, S))
                                                                           : redot(S, P) + redot(F1, F0);
                    if (acc_on) kahan_add(accP[r], cmpP[r], term);
                    if (R > 0) prevP[r] = cmul(S, th);
                }
                if (R > 0 && !psi_one) th = cmul(th, psi);
            }
        }
        if constexpr (SPECTRA) continue;
        // partial sums of this (template, weight, chunk) row for the coset's bins, staged
        // through Y (the last transform's reads of Y ended before its second barrier)
        __syncthreads();
        float* accm = (float*)Y;
#pragma unroll
        for (int r = 0; r < SLP; ++r)
            if (tid + NSL * r <= q.mmax) accm[tid + NSL * r] = accP[r];
        __syncthreads();
        const int o = __ldg(p.coset4_off + c), nbc = __ldg(p.coset4_off + c + 1) - o;
        float* outp = raw + ((size_t)t * 2 * q.n_chunks + (size_t)w * q.n_chunks + chunk) * p.N_f;
        for (int i = tid; i < nbc; i += TT_THREADS) outp[__ldg(p.coset4_k + o + i)] = accm[__ldg(p.coset4_m + o + i)];
        // the next unit's first pass rewrites Y: the unit fetch's barrier orders it
    }
}

// Fold of a long segment (N_s > L) onto the L = 4096 positions of the coset transforms
// (Sec. III B 4 with a segment longer than the on-chip transform): position p of coset c
// takes sum_f x[p + f L] W_N^((b0+c)(p + f L)) = W_N^((b0+c) p) Z_q[p] with
// Z_q[p] = sum_f x[p + f L] W_C^(q f) and q = (b0 + c) mod C (W_N^L = W_C), a C-point
// DFT over the fold index f computed once per (template, detector, weight, segment) for
// every q, instead of each coset re-reading and re-twiddling the whole segment.  The
// persistent kernel applies W_N^((b0+c) p) as it does for whole segments.
// grid: x = segment K, y = detector X * 2 + weight w, z = template of the batch.
// ab: [n_t][Q][2][N_tau], z: [n_t][Q][2][M][C][L] (both in the plan's storage type).
template <bool BF16>
__global__ void __launch_bounds__(TT_THREADS)
fold_kernel(DevParams p, const void* __restrict__ ab, const float4* __restrict__ norm, void* __restrict__ z) {
    __shared__ float2 wc[FOLD_MAX_C];   // W_C^n
    constexpr int L = TT_L;
    const int64_t K = blockIdx.x;
    const int X = blockIdx.y >> 1, w = blockIdx.y & 1;
    const int64_t t = blockIdx.z;
    const int Q = p.Q, C = p.C4, tid = threadIdx.x;
    const int64_t N_s = p.N_s, M = p.M;
    const float4 nm = norm[((size_t)t * Q + X) * M + K];
    if (!(nm.x + nm.y > 0.f)) return;   // no weight in the segment: the row is never read
    for (int n = tid; n < C; n += TT_THREADS) {
        float sn, cs;
        sincospif(-2.0f * (float)n / (float)C, &sn, &cs);
        wc[n] = make_float2(cs, sn);
    }
    __syncthreads();
    const int F = (int)((N_s + L - 1) / L);
    const size_t row = (((size_t)t * Q + X) * 2 + w) * p.N_tau + (size_t)(K * N_s);
    const size_t zrow = ((((size_t)t * Q + X) * 2 + w) * M + K) * C * L;
    for (int i = 0; i < L / TT_THREADS; ++i) {
        const int pp = tid + TT_THREADS * i;
        float2 a[FOLD_MAX_F];
#pragma unroll
        for (int f = 0; f < FOLD_MAX_F; ++f) {
            const int64_t sidx = pp + (int64_t)f * L;
            a[f] = make_float2(0.f, 0.f);
            if (f < F && sidx < N_s) {
                if constexpr (BF16) a[f] = __bfloat1622float2(((const __nv_bfloat162*)ab)[row + sidx]);
                else a[f] = __ldg((const float2*)ab + row + sidx);
            }
        }
        for (int qq = 0; qq < C; ++qq) {
            float2 acc = a[0];
#pragma unroll
            for (int f = 1; f < FOLD_MAX_F; ++f)
                if (f < F) acc = cadd(acc, cmul(a[f], wc[(qq * f) & (C - 1)]));
            const size_t o = zrow + (size_t)qq * L + pp;
            if constexpr (BF16) ((__nv_bfloat162*)z)[o] = __float22bfloat162_rn(acc);
            else ((float2*)z)[o] = acc;
        }
    }
}

// fold_kernel for C = 64 cosets (the long-lag band: N_FFT = 2^18 = 64 x 4096) and at most
// 16 folds, by a radix-8 split of the 64-point DFT over the fold index: with q = u + 8 v
// and f = f1 + 8 f2, W_64^(q f) = W_8^(v f1) W_64^(u f1) W_8^(u f2), so
// Z_(u+8v) = DFT8_v[ W_64^(u f1) (a_(f1) + a_(f1+8) W_8^u) ]: per residue u a twiddle and
// one register 8-point DFT instead of 64 x F products.
template <bool BF16, int MAXF>
__global__ void __launch_bounds__(TT_THREADS, 3)
fold64_kernel(DevParams p, const void* __restrict__ ab, const float4* __restrict__ norm, void* __restrict__ z) {
    static_assert(MAXF > 8 && MAXF <= 16, "folds f = f1 + 8 f2 with f2 < 2");
    __shared__ float2 w64[64];   // W_64^n = W_4096^(64 n)
    constexpr int L = TT_L, C = 64;
    const int64_t K = blockIdx.x;
    const int X = blockIdx.y >> 1, w = blockIdx.y & 1;
    const int64_t t = blockIdx.z;
    const int Q = p.Q, tid = threadIdx.x;
    const int64_t N_s = p.N_s, M = p.M;
    const float4 nm = norm[((size_t)t * Q + X) * M + K];
    if (!(nm.x + nm.y > 0.f)) return;   // no weight in the segment: the row is never read
    if (tid < C) w64[tid] = __ldg(p.twL + 64 * tid);
    __syncthreads();
    const int F = (int)((N_s + L - 1) / L);
    const size_t row = (((size_t)t * Q + X) * 2 + w) * p.N_tau + (size_t)(K * N_s);
    const size_t zrow = ((((size_t)t * Q + X) * 2 + w) * M + K) * C * L;
    for (int i = 0; i < L / TT_THREADS; ++i) {
        const int pp = tid + TT_THREADS * i;
        float2 a[MAXF];
#pragma unroll
        for (int f = 0; f < MAXF; ++f) {
            const int64_t sidx = pp + (int64_t)f * L;
            a[f] = make_float2(0.f, 0.f);
            if (f < F && sidx < N_s) {
                if constexpr (BF16) a[f] = __bfloat1622float2(((const __nv_bfloat162*)ab)[row + sidx]);
                else a[f] = __ldg((const float2*)ab + row + sidx);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            float2 v[16];
#pragma unroll
            for (int f1 = 0; f1 < 8; ++f1) {
                float2 b = a[f1];
                if (f1 + 8 < MAXF && f1 + 8 < F) b = cadd(b, u == 0 ? a[f1 + 8] : cmul(a[f1 + 8], w64[8 * u]));
                v[f1] = (u == 0 || f1 == 0) ? b : cmul(b, w64[(u * f1) & 63]);
            }
            dft8(v);   // v[j] = sum_f1 W_8^(j f1) (...): Z_(u + 8 j)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const size_t o = zrow + (size_t)(u + 8 * j) * L + pp;
                if constexpr (BF16) ((__nv_bfloat162*)z)[o] = __float22bfloat162_rn(v[j]);
                else ((float2*)z)[o] = v[j];
            }
        }
    }
}

size_t al128(size_t b) { return (b + 127) & ~(size_t)127; }

bool tma_layout(const cc_plan* plan, TmaWork* q, size_t* bytes) {
    const DevParams& p = plan->dp;
    const int esz = p.store == CC_STORE_BF16 ? 4 : 8;
    q->mmax = p.C4 > 0 ? (int)((plan->kbar.back() - plan->k0) / p.C4) : TT_L;
    q->folded = p.N_s > TT_L ? 1 : 0;
    q->n_in = q->folded ? TT_L : (int)p.N_s;
    q->stage_bytes = (uint32_t)(q->n_in * esz);
    size_t o = 0;
    q->off_stage = (uint32_t)o;
    o = al128(o + q->stage_bytes);
    q->off_y = (uint32_t)o;
    o = al128(o + (size_t)padded_len(TT_L) * sizeof(float2));
    q->off_z = (uint32_t)o;
    o = al128(o + (size_t)padded_len(TT_L) * sizeof(float2));
    q->off_h = (uint32_t)o;
    o = al128(o + (size_t)(q->mmax + 1) * sizeof(float2));
    q->off_bar = (uint32_t)o;
    o += 16;
    *bytes = o;
    return o <= 113 * 1024;   // two CTAs per SM
}

template <bool BF16, bool SPECTRA>
int occupancy(size_t smem) {
    int n = 0;
    if (cudaFuncSetAttribute(segpair_tma_kernel<BF16, SPECTRA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, segpair_tma_kernel<BF16, SPECTRA>, TT_THREADS, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

}  // namespace

// Coset length 4096, segments of an even number of samples (a multiple of 4 with BF16
// storage: rows then start on 16-byte boundaries for the bulk copies), Q <= 2, R <= 1, the
// output bins in the lower half of each coset transform; segments longer than 4096
// samples are folded first (at most FOLD_MAX_F folds and FOLD_MAX_C cosets).
bool segpair_tma_supported(const cc_plan* plan) {
    const DevParams& p = plan->dp;
    const bool padded = p.L < TT_L && plan->tuning.transform_len == TT_L && p.C4 > 0;   // N_s <= L < 4096
    if ((p.L != TT_L && !padded) || p.Q > 2 || p.R > 1 || p.pair_mode == CC_PAIRS_CROSS_ONLY || plan->N_f < 1)
        return false;
    if (p.N_s > TT_L && (p.C4 > FOLD_MAX_C || (p.N_s + TT_L - 1) / TT_L > FOLD_MAX_F)) return false;
    // rows start on 16-byte boundaries for the bulk copies
    if (p.N_s % (p.store == CC_STORE_BF16 ? 4 : 2)) return false;
    TmaWork q;
    size_t bytes;
    if (!tma_layout(plan, &q, &bytes)) return false;
    return 2 * q.mmax < TT_L;
}

// Segment chunks per (template, weight) for a batch of n_t templates: about
// `units per CTA` (the tuning's chunk_waves, default 24) units per persistent CTA, each
// chunk at least 4R + 1 segments.
int segpair_tma_chunks(const cc_plan* plan, int64_t n_t) {
    const DevParams& p = plan->dp;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t per_cta = plan->tuning.chunk_waves > 0 ? plan->tuning.chunk_waves : 24;
    const int64_t ctas_per_coset = std::max<int64_t>(1, 2 * (int64_t)sms / p.C4);
    const int64_t want = (per_cta * ctas_per_coset + 2 * n_t - 1) / (2 * n_t);
    const int64_t maxch = std::max<int64_t>(1, p.M / (4 * p.R + 1));
    return (int)std::max<int64_t>(1, std::min<int64_t>({want, maxch, 32767}));
}

bool segpair_tma_folded(const cc_plan* plan) { return plan->dp.N_s > TT_L; }

// Bytes of the fold kernel's output per template (0 for whole segments).
size_t segpair_tma_fold_bytes(const cc_plan* plan) {
    if (!segpair_tma_folded(plan)) return 0;
    const DevParams& p = plan->dp;
    return (size_t)p.Q * 2 * p.M * p.C4 * TT_L * (p.store == CC_STORE_BF16 ? 4 : 8);
}

cc_status launch_fold(cc_plan* plan, int64_t n_t, const void* ab, const float4* norm, void* z, cudaStream_t st) {
    const DevParams& p = plan->dp;
    if (n_t > 65535 || p.M > 0x7fffffff) return fail(CC_ERR_UNSUPPORTED, "fold launch size");
    const dim3 grid((unsigned)p.M, (unsigned)(2 * p.Q), (unsigned)n_t);
    const bool bf16 = p.store == CC_STORE_BF16;
    const int64_t F = (p.N_s + TT_L - 1) / TT_L;
    if (p.C4 == 64 && F <= 9) {   // the long-lag band: nine folds
        if (bf16) fold64_kernel<true, 9><<<grid, TT_THREADS, 0, st>>>(p, ab, norm, z);
        else fold64_kernel<false, 9><<<grid, TT_THREADS, 0, st>>>(p, ab, norm, z);
    } else if (p.C4 == 64) {
        if (bf16) fold64_kernel<true, 16><<<grid, TT_THREADS, 0, st>>>(p, ab, norm, z);
        else fold64_kernel<false, 16><<<grid, TT_THREADS, 0, st>>>(p, ab, norm, z);
    } else {
        if (bf16) fold_kernel<true><<<grid, TT_THREADS, 0, st>>>(p, ab, norm, z);
        else fold_kernel<false><<<grid, TT_THREADS, 0, st>>>(p, ab, norm, z);
    }
    count_launch();
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "fold launch");
}

cc_status launch_segpair_tma(cc_plan* plan, const SegPairLayout& lay, int64_t n_t, const void* ab,
                             const float4* norm, float* raw, int* counters, cudaStream_t st) {
    const DevParams& p = plan->dp;
    TmaWork q;
    size_t bytes;
    if (!tma_layout(plan, &q, &bytes)) return fail(CC_ERR_UNSUPPORTED, "segpair_tma layout");
    q.n_chunks = lay.n_chunks;
    q.chunk_len = lay.chunk_len;
    q.units = n_t * 2 * lay.n_chunks;
    if (q.units > 0x7fffffff) return fail(CC_ERR_UNSUPPORTED, "too many work units in one launch");
    const bool bf16 = p.store == CC_STORE_BF16;
    const int occ = bf16 ? occupancy<true, false>(bytes) : occupancy<false, false>(bytes);
    if (occ < 1) return fail(CC_ERR_UNSUPPORTED, "segpair_tma kernel does not fit an SM");
    int dev = 0, sms = 152;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attributes");
    const int64_t grid = std::min<int64_t>((int64_t)occ * sms, q.units * p.C4);
    if ((e = cudaMemsetAsync(counters, 0, sizeof(int) * p.C4, st)) != cudaSuccess)
        return cuda_fail(e, "unit counters");
    if (bf16)
        segpair_tma_kernel<true, false><<<(unsigned)grid, TT_THREADS, bytes, st>>>(p, q, ab, norm, raw, counters,
                                                                                  nullptr);
    else
        segpair_tma_kernel<false, false><<<(unsigned)grid, TT_THREADS, bytes, st>>>(p, q, ab, norm, raw, counters,
                                                                                   nullptr);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "segpair_tma launch");
    return CC_OK;
}

// The staged segment-FFT stage by the persistent kernel: whole segments (N_s <= 4096, even;
// a multiple of 4 with BF16 storage) on 4096-point cosets (the plan's own, or zero-padded
// when the plan is tuned to transform_len 4096), Q <= 2, output bins in the lower half of
// each coset transform.
bool segfft_tma_supported(const cc_plan* plan) {
    const DevParams& p = plan->dp;
    const bool padded = p.L < TT_L && plan->tuning.transform_len == TT_L && p.C4 > 0;
    if ((p.L != TT_L && !padded) || p.Q > 2 || p.N_s > TT_L || plan->N_f < 1) return false;
    if (p.N_s % (p.store == CC_STORE_BF16 ? 4 : 2)) return false;
    TmaWork q;
    size_t bytes;
    if (!tma_layout(plan, &q, &bytes)) return false;
    return 2 * q.mmax < TT_L;
}

cc_status launch_segfft_tma(cc_plan* plan, int64_t n_t, const void* ab, float2* F, int* counters, cudaStream_t st) {
    const DevParams& p = plan->dp;
    TmaWork q;
    size_t bytes;
    if (!tma_layout(plan, &q, &bytes)) return fail(CC_ERR_UNSUPPORTED, "segpair_tma layout");
    const bool bf16 = p.store == CC_STORE_BF16;
    const int occ = bf16 ? occupancy<true, true>(bytes) : occupancy<false, true>(bytes);
    if (occ < 1) return fail(CC_ERR_UNSUPPORTED, "segpair_tma kernel does not fit an SM");
    int dev = 0, sms = 152;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device attributes");
    // chunks of segments: about 24 units per persistent CTA
    const int64_t ctas_per_coset = std::max<int64_t>(1, (int64_t)occ * sms / p.C4);
    const int64_t n_chunks = std::max<int64_t>(1, std::min<int64_t>({(24 * ctas_per_coset + 2 * n_t - 1) / (2 * n_t),
                                                                     p.M, 32767}));
    q.n_chunks = (int)n_chunks;
    q.chunk_len = (p.M + n_chunks - 1) / n_chunks;
    q.units = n_t * 2 * n_chunks;
    if (q.units > 0x7fffffff) return fail(CC_ERR_UNSUPPORTED, "too many work units in one launch");
    const int64_t grid = std::min<int64_t>((int64_t)occ * sms, q.units * p.C4);
    if ((e = cudaMemsetAsync(counters, 0, sizeof(int) * p.C4, st)) != cudaSuccess)
        return cuda_fail(e, "unit counters");
    if (bf16)
        segpair_tma_kernel<true, true><<<(unsigned)grid, TT_THREADS, bytes, st>>>(p, q, ab, nullptr, nullptr,
                                                                                 counters, F);
    else
        segpair_tma_kernel<false, true><<<(unsigned)grid, TT_THREADS, bytes, st>>>(p, q, ab, nullptr, nullptr,
                                                                                  counters, F);
    count_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "segment FFT (persistent) launch");
}

}  // namespace cc
