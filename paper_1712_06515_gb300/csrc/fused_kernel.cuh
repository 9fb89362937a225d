// Fused resample -> segment spectra -> pair sum, without materialising a_r, b_r or F.
//
// One thread-block cluster of CL CTAs handles one (template, chunk of segments).
// For every segment K:
//   * each CTA computes the FP64 timing knots it owns (knot index = rank mod CL) for
//     segment K+1 and resamples its 1/CL slice of segment K (windowed-sinc, heterodyne
//     and f_r* phase, antenna/noise weights) into shared memory;
//   * after one cluster barrier every CTA gathers the whole segment from its peers'
//     shared memory (distributed shared memory), applies the coset twiddle and places
//     sample r at position r mod L of an L-point transform (the segment-start phase
//     Phi_in then falls out of the transform).  The two halves of the CTA (256 threads
//     each) transform two detectors at once: the gather lands in the registers of the
//     first radix-16 Stockham pass, later passes go through a padded buffer per half;
//   * the coset's output bins update the pair sum held on chip: a running sum over
//     detectors of the current segment and a ring of the R previous segments' sums.
// Slices, knot delays and norm partials are double-buffered, so one cluster barrier
// per segment suffices.  Chunks start R segments early to fill the ring; their partial
// sums and normalisations are combined by finalize_kernel.
#pragma once

#include <cooperative_groups.h>
#include <math.h>

#include "common.cuh"
#include "fft_reg.cuh"

namespace cg = cooperative_groups;

namespace cc {

__device__ __forceinline__ const float2* slice_ptr(const FusedLayout& lay, unsigned char* base, int buf,
                                                   int Q, int X, int w) {
    return (const float2*)(base + lay.off_slice) + (((size_t)buf * Q + X) * 2 + w) * lay.S;
}

static_assert(KNOT == 128, "slice blocks and knot indices use shifts by 7");

// barrier of one 256-thread half of the CTA (named barrier 1 or 2)
struct HalfSync {
    int id;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory");
    }
};

// LT: coset transform length (compile-time); PREKNOTS: knot records come from the
// pre-pass (global memory) instead of being computed and exchanged in the cluster;
// REGPAIR: the pair sum is formed in registers straight from the last FFT pass (one
// coset per CTA, Q <= 2, R <= 1, no cross-only pair set, bins in the lower half of the
// coset transform).
template <int LT, bool PREKNOTS, bool REGPAIR>
__global__ void __launch_bounds__(FUSED_THREADS, 1)
fused_kernel(DevParams p, FusedLayout lay, const cc_template* __restrict__ tm, int64_t t_base,
             float* __restrict__ raw_out, double* __restrict__ dpart_out,
             const KnotRec* __restrict__ kn, int64_t nkn) {
    extern __shared__ __align__(16) unsigned char sm[];
    static_assert(LT >= 64 && LT <= 4096, "coset length");
    constexpr int L = LT;
    const int CL = lay.CL;
    const int rank = (int)cg::this_cluster().block_rank();
    const int chunk = blockIdx.y;
    const int64_t t = t_base + blockIdx.z;
    const int Q = p.Q, nb = lay.nb;
    const int64_t N_s = p.N_s, R = p.R;
    const int64_t Ka = (int64_t)chunk * lay.chunk_len;
    const int64_t Kb = imin64(p.M, Ka + lay.chunk_len);
    const int64_t Kl = imax64(0, Ka - R);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncos = (p.C + CL - 1 - rank) / CL;   // cosets c = rank, rank + CL, ...

    float2* fftb = (float2*)(sm + lay.off_fft);
    float2* ring = (float2*)(sm + lay.off_ring);
    float2* same = (float2*)(sm + lay.off_same);
    float* rho = (float*)(sm + lay.off_rho);
    float* comp = rho + nb;
    double* dkb = (double*)(sm + lay.off_dk);
    KnotRec* recb = (KnotRec*)(sm + lay.off_rec);
    float* wpart = (float*)(sm + lay.off_wpart);
    float4* nring = (float4*)(sm + lay.off_nring);
    int2* bins = (int2*)(sm + lay.off_bins);
    // [SEGACT_DEPTH][CC_MAX_DET]: detector has weight in segment K (slot (K - Kl) mod depth)
    int* segact = (int*)(sm + lay.off_flags);
    int* cstart = (int*)(bins + nb);

    const Orbit orb = make_orbit(p, tm[t]);

    // this CTA's bins: cosets rank, rank+CL, ... concatenated
    if (tid == 0) {
        int acc = 0;
        for (int j = 0; j < ncos; ++j) {
            cstart[j] = acc;
            const int c = rank + j * CL;
            acc += __ldg(p.coset_off + c + 1) - __ldg(p.coset_off + c);
        }
        cstart[ncos] = acc;
    }
    __syncthreads();
    const int nmine = cstart[ncos];
    for (int j = 0; j < ncos; ++j) {
        const int c = rank + j * CL;
        const int o = __ldg(p.coset_off + c), n = __ldg(p.coset_off + c + 1) - o;
        for (int i = tid; i < n; i += FUSED_THREADS)
            bins[cstart[j] + i] = make_int2(__ldg(p.coset_m + o + i), __ldg(p.coset_k + o + i));
    }
    const int64_t nslot = lay.ring_q > 1 ? R + 1 : R;   // per-detector rings keep one spare slot
    const int ringn = (R > 0 && !REGPAIR) ? (int)nslot * lay.ring_q * 2 * nb : 0;
    for (int i = tid; i < ringn; i += FUSED_THREADS) ring[i] = make_float2(0.f, 0.f);
    if (!lay.regacc)
        for (int i = tid; i < nb; i += FUSED_THREADS) rho[i] = comp[i] = 0.f;
    // with one coset per CTA and at most ACC_SLOTS * FUSED_THREADS bins, thread tid owns
    // bins tid + s FUSED_THREADS and keeps their compensated sums in registers
    float rhoR[ACC_SLOTS], compR[ACC_SLOTS];
#pragma unroll
    for (int s2 = 0; s2 < ACC_SLOTS; ++s2) rhoR[s2] = compR[s2] = 0.f;
    // REGPAIR: thread lt of half w holds, for its outputs m = lt + NSL r (r < SLP) of the
    // coset transform, the weight-w pair sum (compensated) and the previous segment's
    // detector sum of spectra (absolute phase)
    constexpr int RLAST = last_radix(LT);
    constexpr int NSL = LT / RLAST;
    constexpr int SLP = RLAST / 2 > 0 ? RLAST / 2 : 1;
    float accP[SLP], cmpP[SLP];
    float2 prevP[SLP];
#pragma unroll
    for (int s2 = 0; s2 < SLP; ++s2) {
        accP[s2] = cmpP[s2] = 0.f;
        prevP[s2] = make_float2(0.f, 0.f);
    }
    if (tid < (int)(R + 1) * Q) nring[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    double Dacc = 0.0;

    auto knot_range = [&](int64_t K, int64_t* kA) {
        const int64_t seg0 = K * N_s;
        *kA = floor_div(seg0, KNOT) - 1;
        return (int)(floor_div(seg0 + N_s - 1, KNOT) + 2 - *kA + 1);
    };
    // FP64 knot delays owned by this CTA for segment K into buffer `buf`
    auto compute_knots = [&](int64_t K, int buf) {
        int64_t kA;
        const int nk = knot_range(K, &kA);
        const int nown = (nk - rank + CL - 1) / CL;
        // the block's last threads carry the lightest resampling share, so the FP64
        // chains start there and overlap the others' FP32 work
        for (int j = FUSED_THREADS - 1 - tid; j < nown * Q && j >= 0; j += FUSED_THREADS) {
            const int X = j / nown, i = rank + (j % nown) * CL;
            dkb[((size_t)buf * Q + X) * lay.nkseg + i] =
                knot_delay(p, X, orb, (double)((kA + i) * KNOT) * p.dt);
        }
    };
    auto remote_dk = [&](int buf, int X, int i) -> double {
        const double* b = dkb + ((size_t)buf * Q + X) * lay.nkseg + i;
        return *cg::this_cluster().map_shared_rank(b, i % CL);
    };
    // Slices are dealt in blocks of KNOT samples: segment-local block q belongs to CTA
    // q mod CL and sits at local block q / CL.  A block spans at most two knots.
    const int nblk = (int)((N_s + KNOT - 1) / KNOT);
    const int nmyb = (nblk - rank + CL - 1) / CL;
    // knot records of this CTA's blocks of segment K from the cluster's knot delays
    auto build_records = [&](int64_t K, int buf) {
        int64_t kA;
        knot_range(K, &kA);
        const int64_t seg0 = K * N_s, seg1 = seg0 + N_s;
        for (int j = tid; j < 2 * nmyb * Q; j += FUSED_THREADS) {
            const int X = j / (2 * nmyb), jj = j % (2 * nmyb);
            const int qi = jj >> 1, e = jj & 1;
            const int64_t r0 = seg0 + (int64_t)(qi * CL + rank) * KNOT;
            const int64_t r1 = imin64(r0 + KNOT, seg1);
            const int64_t k = (r0 >> 7) + e;
            if (k > ((r1 - 1) >> 7)) continue;
            const int i = (int)(k - kA);
            recb[((size_t)buf * Q + X) * lay.nrec + jj] =
                make_knot(p, remote_dk(buf, X, i - 1), remote_dk(buf, X, i), remote_dk(buf, X, i + 1),
                          remote_dk(buf, X, i + 2), (double)(k * KNOT) * p.dt);
        }
    };
    auto cluster_sync = [&]() { cg::this_cluster().sync(); };

    // Gap skipping (knot records from the pre-pass): the detector times t = r - d of
    // segment K lie within [seg0 - max d - 2, seg1 + 2 - min d] (d from the segment's
    // knots; the cubic between knots stays within 1e-4 samples of them); a detector
    // whose noise blocks there are all gaps has zero weight in the whole segment, so its
    // resampling and transforms are skipped and it contributes F = 0.  Called by warp X.
    auto seg_active = [&](int64_t K, int X) -> int {
        if constexpr (!PREKNOTS) return 1;
        const KnotRec* __restrict__ knX = kn + ((size_t)blockIdx.z * Q + X) * nkn;
        const int64_t s0 = K * N_s, s1 = s0 + N_s;
        const int64_t ka = s0 >> 7, kb = imin64(((s1 - 1) >> 7) + 1, nkn - 1);
        float dmin = 3.0e38f, dmax = -3.0e38f;
        for (int64_t k = ka + lane; k <= kb; k += 32) {
            const KnotRec kr = load_knot(knX + k);
            const float d = (float)kr.N + kr.f;
            dmin = fminf(dmin, d);
            dmax = fmaxf(dmax, d);
        }
        for (int o = 16; o > 0; o >>= 1) {
            dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
            dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        }
        const int tlo = (int)s0 - (int)ceilf(dmax) - 2, thi = (int)s1 - (int)floorf(dmin) + 2;
        int blo = floor_div32(tlo, p.nsft), bhi = floor_div32(thi, p.nsft);
        const int ns = (int)p.n_sig[X];
        blo = blo < 0 ? 0 : blo;
        bhi = bhi > ns - 1 ? ns - 1 : bhi;
        if (blo > bhi) return 0;
        return __ldg(p.lockc[X] + bhi + 1) - __ldg(p.lockc[X] + blo) > 0 ? 1 : 0;
    };
    // Flags are written two segments ahead (by warp X, after the cluster barrier of
    // segment K for segment K + 2) so that a cluster barrier always separates a flag's
    // write from its reads: the two halves of a CTA meet at no other barrier.
    if (warp < Q) {
        for (int64_t K = Kl; K < imin64(Kl + 2, Kb); ++K) {
            const int a = seg_active(K, warp);
            if (lane == 0) segact[(int)((K - Kl) & (SEGACT_DEPTH - 1)) * CC_MAX_DET + warp] = a;
        }
    }
    __syncthreads();

    // prologue: knots and records of the first segment
    if constexpr (!PREKNOTS) {
        compute_knots(Kl, 0);
        cluster_sync();
        build_records(Kl, 0);
        __syncthreads();
    }

    for (int64_t K = Kl; K < Kb; ++K) {
        const int b = (int)((K - Kl) & 1);
        const int sa_slot = (int)((K - Kl) & (SEGACT_DEPTH - 1));
        const int64_t seg0 = K * N_s;
        // (1) knot delays of the next segment (FP64, a few threads)
        if constexpr (!PREKNOTS)
            if (K + 1 < Kb) compute_knots(K + 1, b ^ 1);
        // (2) resample this CTA's blocks of segment K for every detector
        {
            const int nloc = nmyb * KNOT;
            for (int X = 0; X < Q; ++X) {
                float A = 0.f, B = 0.f, Cn = 0.f;
                const bool actX = segact[sa_slot * CC_MAX_DET + X] != 0;
                const float2* __restrict__ x = p.x[X];
                float2* sa = (float2*)slice_ptr(lay, sm, b, Q, X, 0);
                float2* sb = (float2*)slice_ptr(lay, sm, b, Q, X, 1);
                const KnotRec* rec = recb + ((size_t)b * Q + X) * lay.nrec;
                const KnotRec* __restrict__ knX = kn + ((size_t)blockIdx.z * Q + X) * nkn;
                for (int li = tid; li < (actX ? nloc : 0); li += FUSED_THREADS) {
                    const int qi = li >> 7;
                    const int rr = (qi * CL + rank) * KNOT + (li & (KNOT - 1));
                    if (rr >= (int)N_s) continue;
                    const int r = (int)seg0 + rr;
                    const int k = r >> 7;
                    KnotRec kr;
                    if constexpr (PREKNOTS) {
                        kr = load_knot(knX + k);
                    } else {
                        const int r0 = (int)seg0 + (qi * CL + rank) * KNOT;
                        kr = rec[2 * qi + (k - (r0 >> 7))];
                    }
                    const SampleTiming st = sample_timing(p, kr, r, k * KNOT);
                    const float2 xv = interp_sample(p, x, st.jstar, st.delta);
                    const float2 xr = cmul(xv, phase_rot(st.psi));
                    const SampleWeights wt = sample_weights(p, X, st.jstar, st.delta);
                    sa[li] = cscale(xr, wt.alpha);
                    sb[li] = cscale(xr, wt.beta);
                    A = fmaf(wt.alpha * wt.alpha, wt.s2, A);
                    B = fmaf(wt.beta * wt.beta, wt.s2, B);
                    Cn = fmaf(wt.alpha * wt.beta, wt.s2, Cn);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    A += __shfl_xor_sync(0xffffffffu, A, o);
                    B += __shfl_xor_sync(0xffffffffu, B, o);
                    Cn += __shfl_xor_sync(0xffffffffu, Cn, o);
                }
                if (lane == 0) {
                    float* wp = wpart + (((size_t)b * FUSED_WARPS + warp) * Q + X) * 4;
                    wp[0] = A;
                    wp[1] = B;
                    wp[2] = Cn;
                }
            }
        }
        cluster_sync();
        // (3) knot records of the next segment's slice
        if constexpr (!PREKNOTS)
            if (K + 1 < Kb) build_records(K + 1, b ^ 1);
        if (K + 2 < Kb && warp < Q) {
            const int a = seg_active(K + 2, warp);
            if (lane == 0) segact[(int)((K + 2 - Kl) & (SEGACT_DEPTH - 1)) * CC_MAX_DET + warp] = a;
        }
        // (4) segment norms and the normalisation (rank 0 holds D): one thread per
        //     (peer, detector, component) sums that peer's warp partials
        if (rank == 0) {
            float* nsum = wpart + (size_t)2 * FUSED_WARPS * Q * 4;   // [CL][Q][3] scratch
            if (tid < CL * Q * 3) {
                const int rr = tid / (Q * 3), X = (tid / 3) % Q, i = tid % 3;
                const float* wp = wpart + (size_t)b * FUSED_WARPS * Q * 4;
                wp = cg::this_cluster().map_shared_rank(wp, rr);
                float v[FUSED_WARPS];
#pragma unroll
                for (int wv = 0; wv < FUSED_WARPS; ++wv) v[wv] = wp[(wv * Q + X) * 4 + i];
                float sacc = 0.f;
#pragma unroll
                for (int wv = 0; wv < FUSED_WARPS; ++wv) sacc += v[wv];
                nsum[tid] = sacc;
            }
            __syncthreads();
            if (tid == 0) {
                float4 nK[CC_MAX_DET];
                for (int X = 0; X < Q; ++X) {
                    float sv[3] = {0.f, 0.f, 0.f};
                    for (int rr = 0; rr < CL; ++rr)
                        for (int i = 0; i < 3; ++i) sv[i] += nsum[(rr * Q + X) * 3 + i];
                    nK[X] = make_float4(sv[0], sv[1], sv[2], 0.f);
                }
                if (K >= Ka) {
                    for (int Y = 0; Y < Q; ++Y) {
                        double sY = 0.0;
                        for (int X = 0; X < Y; ++X)
                            sY += (double)nK[X].x * nK[Y].x + (double)nK[X].y * nK[Y].y +
                                  2.0 * (double)nK[X].z * nK[Y].z;
                        for (int64_t Lg = imax64(0, K - R); Lg < K; ++Lg)
                            for (int X = 0; X < Q; ++X) {
                                if (p.pair_mode == CC_PAIRS_CROSS_ONLY && X == Y) continue;
                                const float4 nl = nring[(Lg % R) * Q + X];
                                sY += (double)nl.x * nK[Y].x + (double)nl.y * nK[Y].y +
                                      2.0 * (double)nl.z * nK[Y].z;
                            }
                        if (p.pair_mode == CC_PAIRS_ALL_ORDERED)
                            sY = 2.0 * sY + (double)nK[Y].x * nK[Y].x + (double)nK[Y].y * nK[Y].y +
                                 2.0 * (double)nK[Y].z * nK[Y].z;
                        Dacc += sY;
                    }
                }
                if (R > 0)
                    for (int X = 0; X < Q; ++X) nring[(K % R) * Q + X] = nK[X];
            }
        }
        // (5) spectra of this CTA's cosets and the pair sum.  Half h of the CTA transforms
        //     detector 2g + h of round g; with at most two detectors (one round) each half
        //     transforms both weights into their own buffers and one pass over the bins
        //     updates the pair sum, otherwise every (weight, round) has its own pass.
        const int half = tid >> 8, lt = tid & 255;
        const HalfSync hsync{1 + half};
        constexpr int PL = padded_len(L);
        constexpr int R1 = 16;                // radix of the first pass
        constexpr int B1 = L / R1;
        const int offn = (int)((-seg0) & (int64_t)(L - 1));   // position p holds r - seg0 = (p + offn) mod L
        const int cur = R > 0 ? (int)(K % nslot) : 0;
        const int nround = (Q + 1) / 2;
        const int* act = segact + sa_slot * CC_MAX_DET;
        // gather + first radix-16 pass into registers, stored to `buf` for the later passes
        auto first_pass = [&](int X, int w, float2* buf, const float2* __restrict__ twr) {
            const float2* sbase = slice_ptr(lay, sm, b, Q, X, w);
            if (lt < B1) {
                float2 v[16];
                if (N_s <= L) {
                    float2 vv[16], tw[16];
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        vv[r] = tw[r] = make_float2(0.f, 0.f);
                        const int rr = (lt + r * B1 + offn) & (L - 1);
                        if (rr < (int)N_s) {
                            const int q = rr >> 7;
                            const int owner = q & (CL - 1);
                            const float2* sp = sbase + (((q >> lay.log2CL) << 7) | (rr & (KNOT - 1)));
                            vv[r] = *cg::this_cluster().map_shared_rank(sp, owner);
                            tw[r] = __ldg(twr + rr);
                        }
                    }
#pragma unroll
                    for (int r = 0; r < 16; ++r) v[r] = cmul(vv[r], tw[r]);
                } else {
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        float2 acc = make_float2(0.f, 0.f);
                        for (int rr = (lt + r * B1 + offn) & (L - 1); rr < (int)N_s; rr += L) {
                            const int q = rr >> 7;
                            const int owner = q & (CL - 1);
                            const float2* sp = sbase + (((q >> lay.log2CL) << 7) | (rr & (KNOT - 1)));
                            const float2 vr = *cg::this_cluster().map_shared_rank(sp, owner);
                            acc = cadd(acc, cmul(vr, __ldg(twr + rr)));
                        }
                        v[r] = acc;
                    }
                }
                dft16(v);
#pragma unroll
                for (int r = 0; r < 16; ++r) buf[padi(lt * R1 + r)] = v[r];
            }
            hsync();
        };
        auto transform = [&](int X, int w, float2* buf, const float2* __restrict__ twr) {
            first_pass(X, w, buf, twr);
            stockham_rest_t<L, 16>(buf, lt, p.twL, hsync);
        };
        // pair-sum term of bin i (transform position m) for weight w and round g, with the
        // round's transforms in bufw[hh * PL]; updates the running detector sum and ring
        auto pair_term = [&](int i, int m, int w, int g, const float2* bufw, float2 wseg) -> float {
            float2 sacc = g == 0 ? make_float2(0.f, 0.f) : same[i];
            float term = 0.f;
            for (int hh = 0; hh < 2; ++hh) {
                const int Xh = 2 * g + hh;
                if (Xh >= Q) break;
                const float2 F = act[Xh] ? cmul(bufw[hh * PL + padi(m)], wseg) : make_float2(0.f, 0.f);
                float2 hv = sacc;
                if (R > 0) {
                    if (lay.ring_q == 1) {
                        for (int sl = 0; sl < (int)R; ++sl) hv = cadd(hv, ring[(sl * 2 + w) * nb + i]);
                    } else {
                        for (int sl = 0; sl < (int)nslot; ++sl) {
                            if (sl == cur) continue;
                            for (int X2 = 0; X2 < Q; ++X2)
                                if (X2 != Xh) hv = cadd(hv, ring[((sl * Q + X2) * 2 + w) * nb + i]);
                        }
                        ring[((cur * Q + Xh) * 2 + w) * nb + i] = F;
                    }
                }
                float tX = redot(F, hv);
                if (p.pair_mode == CC_PAIRS_ALL_ORDERED) tX = fmaf(2.f, tX, redot(F, F));
                term += tX;
                sacc = cadd(sacc, F);
            }
            if (g < nround - 1) same[i] = sacc;
            else if (R > 0 && lay.ring_q == 1) ring[(cur * 2 + w) * nb + i] = sacc;
            return term;
        };
        auto accumulate = [&](int s, int i, float term) {
            if (K < Ka) return;
            if (lay.regacc) kahan_add(rhoR[s], compR[s], term);
            else kahan_add(rho[i], comp[i], term);
        };
        if constexpr (REGPAIR) {
            // Half w transforms weight w of both detectors: detector 0 through the buffer,
            // the last detector's last pass into registers; thread lt then owns outputs
            // m = lt + NSL r of both and forms the weight-w pair terms of those bins:
            //   unordered:   Re(conj(S) P) + Re(conj(F_1) F_0)
            //   all ordered: 2 Re(conj(S) P) + |S|^2
            // with S = F_0 + F_1 this segment's detector sum and P the previous segment's
            // (R = 1; zero for R = 0).  The segment phase wseg cancels within a segment
            // and is applied to S once for the next segment.
            const int c = rank;
            const uint64_t N = (uint64_t)p.N_FFT, mask = N - 1;
            const uint64_t bc = ((uint64_t)p.b0 + (uint64_t)c) & mask;
            const float2 wseg = twiddle_N((bc * ((uint64_t)seg0 & mask)) & mask, N);
            const float2* __restrict__ twr = p.twc + (size_t)c * N_s;
            const int w = half;
            float2* buf0 = fftb + (2 * w) * PL;
            float2* buf1 = buf0 + PL;
            const bool a0 = act[0] != 0, al = act[Q - 1] != 0;
            if (Q > 1 && a0) transform(0, w, buf0, twr);
            float2 v[16];
            if (al) {
                first_pass(Q - 1, w, Q > 1 ? buf1 : buf0, twr);
                stockham_rest_keep_t<L, 16>(Q > 1 ? buf1 : buf0, lt, p.twL, hsync, v);
            }
            if (lt < NSL) {
                const float2 wc = make_float2(wseg.x, -wseg.y);
                const bool acc_on = K >= Ka;
#pragma unroll
                for (int r = 0; r < SLP; ++r) {
                    const int m = lt + NSL * r;
                    if (m <= lay.mmax) {
                        const float2 Fl = al ? v[r] : make_float2(0.f, 0.f);
                        float2 F0 = Fl, F1 = make_float2(0.f, 0.f);
                        if (Q > 1) {
                            F0 = a0 ? buf0[padi(m)] : make_float2(0.f, 0.f);
                            F1 = Fl;
                        }
                        const float2 S = cadd(F0, F1);
                        const float2 P = R > 0 ? cmul(prevP[r], wc) : make_float2(0.f, 0.f);
                        const float term = p.pair_mode == CC_PAIRS_ALL_ORDERED
                                               ? fmaf(2.f, redot(S, P), redot(S, S))
                                               : redot(S, P) + redot(F1, F0);
                        if (acc_on) kahan_add(accP[r], cmpP[r], term);
                        if (R > 0) prevP[r] = cmul(S, wseg);
                    }
                }
            }
            // with knots computed in the cluster, the next segment's knot records (built
            // by all threads above) are read by both halves in the next resampling pass
            if constexpr (!PREKNOTS) __syncthreads();
        } else
        for (int j = 0; j < ncos; ++j) {
            const int c = rank + j * CL;
            const uint64_t N = (uint64_t)p.N_FFT, mask = N - 1;
            const uint64_t bc = ((uint64_t)p.b0 + (uint64_t)c) & mask;
            const float2 wseg = twiddle_N((bc * ((uint64_t)seg0 & mask)) & mask, N);
            const float2* __restrict__ twr = p.twc + (size_t)c * N_s;
            const int i0 = cstart[j], i1 = cstart[j + 1];
            if (lay.bothw) {
                if (half < Q && act[half]) {
#pragma unroll 1
                    for (int w = 0; w < 2; ++w) transform(half, w, fftb + (2 * w + half) * PL, twr);
                }
                __syncthreads();
#pragma unroll
                for (int s = 0; s < ACC_SLOTS; ++s) {
                    const int i = i0 + tid + s * FUSED_THREADS;
                    if (s * FUSED_THREADS < i1 - i0 && i < i1) {
                        const int m = bins[i].x;
                        float term = 0.f;
#pragma unroll 1
                        for (int w = 0; w < 2; ++w) term += pair_term(i, m, w, 0, fftb + 2 * w * PL, wseg);
                        accumulate(s, i, term);
                    }
                }
                for (int i = i0 + tid + ACC_SLOTS * FUSED_THREADS; i < i1; i += FUSED_THREADS) {
                    const int m = bins[i].x;
                    float term = 0.f;
#pragma unroll 1
                    for (int w = 0; w < 2; ++w) term += pair_term(i, m, w, 0, fftb + 2 * w * PL, wseg);
                    accumulate(0, i, term);
                }
                __syncthreads();
            } else {
                for (int w = 0; w < 2; ++w) {
                    for (int g = 0; g < nround; ++g) {
                        const int X = 2 * g + half;
                        if (X < Q && act[X]) transform(X, w, fftb + half * PL, twr);
                        __syncthreads();
#pragma unroll
                        for (int s = 0; s < ACC_SLOTS; ++s) {
                            const int i = i0 + tid + s * FUSED_THREADS;
                            if (i < i1) accumulate(s, i, pair_term(i, bins[i].x, w, g, fftb, wseg));
                        }
                        for (int i = i0 + tid + ACC_SLOTS * FUSED_THREADS; i < i1; i += FUSED_THREADS)
                            accumulate(0, i, pair_term(i, bins[i].x, w, g, fftb, wseg));
                        __syncthreads();
                    }
                }
            }
        }
    }
    // every peer may still read this CTA's shared memory until the cluster is done
    cluster_sync();
    float* outp = raw_out + ((size_t)t * lay.n_chunks + chunk) * p.N_f;
    if constexpr (REGPAIR) {
        // the two halves' weight sums meet in shared memory (the transform buffers are free)
        float* accm = (float*)fftb;
        const int lt = tid & 255;
        if (tid < 256 && lt < NSL) {
#pragma unroll
            for (int r = 0; r < SLP; ++r)
                if (lt + NSL * r <= lay.mmax) accm[lt + NSL * r] = accP[r];
        }
        __syncthreads();
        if (tid >= 256 && lt < NSL) {
#pragma unroll
            for (int r = 0; r < SLP; ++r)
                if (lt + NSL * r <= lay.mmax) accm[lt + NSL * r] += accP[r];
        }
        __syncthreads();
        for (int i = tid; i < nmine; i += FUSED_THREADS) outp[bins[i].y] = accm[bins[i].x];
    } else if (lay.regacc) {
#pragma unroll
        for (int s2 = 0; s2 < ACC_SLOTS; ++s2) {
            const int i = tid + s2 * FUSED_THREADS;
            if (i < nmine) outp[bins[i].y] = rhoR[s2];
        }
    } else {
        for (int i = tid; i < nmine; i += FUSED_THREADS) outp[bins[i].y] = rho[i];
    }
    if (rank == 0 && tid == 0) dpart_out[(size_t)t * lay.n_chunks + chunk] = Dacc;
}

// Launch of one instantiation.  The fused_l*.cu translation units instantiate these for
// different coset lengths (compiled in parallel); fused.cu only declares them.
template <int LT>
cudaError_t launch_fused_lt(const cudaLaunchConfig_t& cfg, bool pre, bool regpair, const DevParams& p,
                            const FusedLayout& lay, const cc_template* t_dev, int64_t tb, float* raw,
                            double* dpart, const KnotRec* kn, int64_t nkn) {
    if (pre && regpair)
        return cudaLaunchKernelEx(&cfg, fused_kernel<LT, true, true>, p, lay, t_dev, tb, raw, dpart, kn, nkn);
    if (pre) return cudaLaunchKernelEx(&cfg, fused_kernel<LT, true, false>, p, lay, t_dev, tb, raw, dpart, kn, nkn);
    if (regpair)
        return cudaLaunchKernelEx(&cfg, fused_kernel<LT, false, true>, p, lay, t_dev, tb, raw, dpart, kn, nkn);
    return cudaLaunchKernelEx(&cfg, fused_kernel<LT, false, false>, p, lay, t_dev, tb, raw, dpart, kn, nkn);
}

template <int LT>
const void* fused_kernel_ptr(bool pre, bool regpair) {
    if (pre) return regpair ? (const void*)fused_kernel<LT, true, true> : (const void*)fused_kernel<LT, true, false>;
    return regpair ? (const void*)fused_kernel<LT, false, true> : (const void*)fused_kernel<LT, false, false>;
}

#define CC_FUSED_DECL(PREFIX, LV)                                                                      \
    PREFIX template cudaError_t launch_fused_lt<LV>(const cudaLaunchConfig_t&, bool, bool, const DevParams&, \
                                                    const FusedLayout&, const cc_template*, int64_t, float*, \
                                                    double*, const KnotRec*, int64_t);                  \
    PREFIX template const void* fused_kernel_ptr<LV>(bool, bool);
#define CC_FUSED_INSTANTIATE(LV) CC_FUSED_DECL(, LV)
#define CC_FUSED_EXTERN(LV) CC_FUSED_DECL(extern, LV)

}  // namespace cc
