// Staged path of the crosscorr C ABI: resample -> segment spectra -> pair sum, each
// stage materialising its output in device memory.  Used for per-stage parity and
// per-stage HBM measurement; the fused path (search.cu) shares the device helpers.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "segpair.cuh"
#include "fft_reg.cuh"

namespace cc {

constexpr int RS_THREADS = 256;
constexpr int FFT_THREADS = 256;
constexpr int PAIR_THREADS = 256;
constexpr int64_t MAX_GRID_YZ = 65535;

__device__ __forceinline__ float2 load_series(const void* base, int store, int64_t i) {
    if (store == CC_STORE_BF16) {
        __nv_bfloat162 v = ((const __nv_bfloat162*)base)[i];
        return __bfloat1622float2(v);
    }
    return __ldg((const float2*)base + i);
}

__device__ __forceinline__ void store_series(void* base, int store, int64_t i, float2 v) {
    if (store == CC_STORE_BF16)
        ((__nv_bfloat162*)base)[i] = __float22bfloat162_rn(v);
    else
        ((float2*)base)[i] = v;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// Knots covering segment [seg0, seg0 + N_s): k in [kA, kB] with kA one below the
// first knot and kB two above the last, so every sample has its four knots.
__device__ __forceinline__ void segment_knot_range(const DevParams& p, int64_t seg0, int64_t* kA,
                                                   int64_t* kB) {
    *kA = floor_div(seg0, KNOT) - 1;
    *kB = floor_div(seg0 + p.N_s - 1, KNOT) + 2;
}

// Longest shared-memory window of x a resampling block stages: the segment, the drift
// of the delay across it (|d'| < 2.5e-4 for the Earth and a binary orbit) and the taps.
__host__ __device__ inline int resample_window_len(const DevParams& p) {
    return (int)(p.N_s + p.N_s / 512 + 2 * (p.D > 4 ? p.D : 4) + 48);
}

// Stage 1: one block per (segment K, detector X, template t).  With `kn` (knot records
// of the pre-pass, [n_t][Q][nkn]) the FP64 knots are not recomputed, and a segment whose
// detector times all fall in gaps is skipped: its norms are written as zero and its
// a_r, b_r are written as zero (`write_inactive`, the staged stage: every weight there is
// zero) or left unwritten (the two-pass search reads a segment only when its norms are
// nonzero).  Without `kn` every sample is computed.  The parameter block comes last: with
// it first, the offsets of the small parameters after it moved with its size, and at some
// sizes the two-pass variant compiled to 52 registers instead of 32 and ran 15 % slower.
template <int DT, bool PRE>
__global__ void __launch_bounds__(RS_THREADS)
resample_kernel(const cc_template* __restrict__ tm, int64_t t_base, void* ab, float4* __restrict__ norm,
                const KnotRec* __restrict__ kn, int64_t nkn, int use_window, int write_inactive, DevParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float red[32];
    __shared__ int active;
    const int64_t K = blockIdx.x;
    const int X = blockIdx.y;
    const int64_t t = t_base + blockIdx.z;
    const int64_t seg0 = K * p.N_s;
    const int tid = threadIdx.x;
    int64_t kA, kB;
    segment_knot_range(p, seg0, &kA, &kB);
    const int nk = (int)(kB - kA + 1);
    KnotRec* rec = (KnotRec*)smem;
    float2* xs = (float2*)smem;   // with knot records: the segment's window of x
    __shared__ int win[2];        // first sample and length of the window
    const KnotRec* __restrict__ knX = PRE ? kn + ((size_t)t * p.Q + X) * nkn : nullptr;
    const float2* __restrict__ x = p.x[X];

    if constexpr (PRE) {
        // detector times of the segment lie within [seg0 - max d - 2, seg1 + 2 - min d]
        // (d from the segment's knots; the cubic between knots stays within 1e-4 samples
        // of them); weight only if a noise block there is locked
        if (tid < 32) {
            const int64_t ka = seg0 >> 7, kb = imin64(((seg0 + p.N_s - 1) >> 7) + 1, nkn - 1);
            float dmin = 3.0e38f, dmax = -3.0e38f;
            for (int64_t k = ka + tid; k <= kb; k += 32) {
                const KnotRec kr = load_knot(knX + k);
                const float d = (float)kr.N + kr.f;
                dmin = fminf(dmin, d);
                dmax = fmaxf(dmax, d);
            }
            for (int o = 16; o > 0; o >>= 1) {
                dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
                dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
            }
            if (tid == 0) {
                const int tlo = (int)seg0 - (int)ceilf(dmax) - 2;
                const int thi = (int)(seg0 + p.N_s) - (int)floorf(dmin) + 2;
                int blo = floor_div32(tlo, p.nsft), bhi = floor_div32(thi, p.nsft);
                const int ns = (int)p.n_sig[X];
                blo = blo < 0 ? 0 : blo;
                bhi = bhi > ns - 1 ? ns - 1 : bhi;
                active = blo <= bhi && __ldg(p.lockc[X] + bhi + 1) - __ldg(p.lockc[X] + blo) > 0;
                // stencil centres lie in [tlo + 1, thi - 1]; taps reach max(D, 4) + 1 beyond
                const int margin = (p.D > 4 ? p.D : 4) + 2;
                win[0] = tlo - margin;
                win[1] = use_window ? min(thi + margin - win[0], resample_window_len(p)) : 0;
            }
        }
        __syncthreads();
        if (!active) {
            if (tid == 0) norm[(t * p.Q + X) * p.M + K] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (write_inactive) {
                const int64_t za = ((t * p.Q + X) * 2 + 0) * p.N_tau + seg0, zb = za + p.N_tau;
                for (int i = tid; i < (int)p.N_s; i += blockDim.x) {
                    store_series(ab, p.store, za + i, make_float2(0.f, 0.f));
                    store_series(ab, p.store, zb + i, make_float2(0.f, 0.f));
                }
            }
            return;
        }
        // the segment's window of the series, zero outside [0, N_t)
        const int w0 = win[0], nw = win[1], N = (int)p.N_t;
        for (int i = tid; i < nw; i += blockDim.x) {
            const int j = w0 + i;
            xs[i] = (j >= 0 && j < N) ? __ldg(x + j) : make_float2(0.f, 0.f);
        }
        __syncthreads();
    } else {
        double* dk = (double*)(smem + sizeof(KnotRec) * nk);
        if (tid < nk) {   // FP64: only the threads that own a knot set up the orbit
            const Orbit orb = make_orbit(p, tm[t]);
            for (int i = tid; i < nk; i += blockDim.x)
                dk[i] = knot_delay(p, X, orb, (double)((kA + i) * KNOT) * p.dt);
        }
        __syncthreads();
        for (int i = 1 + tid; i < nk - 2; i += blockDim.x)
            rec[i] = make_knot(p, dk[i - 1], dk[i], dk[i + 1], dk[i + 2], (double)((kA + i) * KNOT) * p.dt);
        __syncthreads();
    }

    const int64_t sa = ((t * p.Q + X) * 2 + 0) * p.N_tau;
    const int64_t sb = sa + p.N_tau;
    float A = 0.f, B = 0.f, Cn = 0.f;
    const int n_s = (int)p.N_s;
    for (int i = tid; i < n_s; i += blockDim.x) {
        const int r = (int)seg0 + i;
        const int k = r >> 7;
        KnotRec kr;
        if constexpr (PRE) kr = load_knot(knX + k);
        else kr = rec[k - kA];
        const SampleTiming st = sample_timing(p, kr, r, k * KNOT);
        const float2 xv = use_window ? interp_sample_window<DT>(p, x, xs, win[0], win[1], st.jstar, st.delta)
                              : interp_sample(p, x, st.jstar, st.delta);
        const float2 xr = cmul(xv, phase_rot(st.psi));
        const SampleWeights w = sample_weights(p, X, st.jstar, st.delta);
        store_series(ab, p.store, sa + r, cscale(xr, w.alpha));
        store_series(ab, p.store, sb + r, cscale(xr, w.beta));
        A = fmaf(w.alpha * w.alpha, w.s2, A);
        B = fmaf(w.beta * w.beta, w.s2, B);
        Cn = fmaf(w.alpha * w.beta, w.s2, Cn);
    }
    A = block_sum(A, red);
    B = block_sum(B, red);
    Cn = block_sum(Cn, red);
    if (tid == 0) norm[(t * p.Q + X) * p.M + K] = make_float4(A, B, Cn, 0.f);
}

// Stage 2: one block per (coset c, segment K, series s = (t*Q + X)*2 + w).
__global__ void __launch_bounds__(FFT_THREADS)
segfft_kernel(DevParams p, const void* ab, int64_t s_base, float2* __restrict__ F) {
    extern __shared__ __align__(16) float2 buf[];
    const int c = blockIdx.x;
    const int64_t K = blockIdx.y;
    const int64_t s = s_base + blockIdx.z;
    const int64_t seg0 = K * p.N_s, seg1 = seg0 + p.N_s;
    const uint64_t N = (uint64_t)p.N_FFT, mask = N - 1;
    const uint64_t bc = ((uint64_t)p.b0 + (uint64_t)c) & mask;
    const int64_t base = s * p.N_tau;
    const int L = p.L;
    for (int pos = threadIdx.x; pos < L; pos += blockDim.x) {
        int64_t off = ((int64_t)pos - seg0) % L;
        if (off < 0) off += L;
        float2 acc = make_float2(0.f, 0.f);
        for (int64_t r = seg0 + off; r < seg1; r += L) {
            const float2 v = load_series(ab, p.store, base + r);
            const uint64_t j = (bc * ((uint64_t)r & mask)) & mask;
            acc = cadd(acc, cmul(v, twiddle_N(j, N)));
        }
        buf[pos] = acc;
    }
    __syncthreads();
    const float2* res = fft_stockham(buf, buf + L, L, p.log2L, p.twL);
    const int64_t tX = s >> 1;
    const int w = (int)(s & 1);
    float2* Fo = F + ((tX * p.M + K) * 2 + w) * p.N_f;
    const int e = __ldg(p.coset_off + c + 1);
    for (int i = __ldg(p.coset_off + c) + threadIdx.x; i < e; i += blockDim.x)
        Fo[__ldg(p.coset_k + i)] = res[__ldg(p.coset_m + i)];
}

// Stage 2 for coset lengths 64..4096: the radix-16 register/shared-memory transform of
// the fused kernels (first pass straight from the series with the coset twiddle, later
// passes in padded shared memory), then the coset's output bins scattered to F.
template <int LT>
__global__ void __launch_bounds__(FFT_THREADS, 2)
segfft_kernel_t(DevParams p, const void* ab, int64_t s_base, float2* __restrict__ F) {
    extern __shared__ __align__(16) float2 buf[];
    constexpr int L = LT, B1 = L / 16;
    const int c = blockIdx.x;
    const int64_t K = blockIdx.y;
    const int64_t s = s_base + blockIdx.z;
    const int tid = threadIdx.x;
    const int64_t seg0 = K * p.N_s;
    const int N_s = (int)p.N_s;
    const size_t row = (size_t)s * p.N_tau + seg0;
    const float2* __restrict__ twr = p.twc + (size_t)c * p.N_s;
    const int offn = (int)((-seg0) & (int64_t)(L - 1));
    auto sync = []() { __syncthreads(); };
    if (tid < B1) {
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            float2 acc = make_float2(0.f, 0.f);
            for (int rr = (tid + r * B1 + offn) & (L - 1); rr < N_s; rr += L)
                acc = cadd(acc, cmul(load_series(ab, p.store, row + rr), __ldg(twr + rr)));
            v[r] = acc;
        }
        dft16(v);
        float2* d = buf + 17 * tid;   // padi(16 tid + r)
#pragma unroll
        for (int r = 0; r < 16; ++r) d[r] = v[r];
    }
    __syncthreads();
    stockham_rest_t<L, 16>(buf, tid, p.twL, sync);
    // the segment-relative twiddles leave out the segment-start phase W_N^((b0 + c) seg0)
    const uint64_t N = (uint64_t)p.N_FFT, mask = N - 1;
    const uint64_t bc = ((uint64_t)p.b0 + (uint64_t)c) & mask;
    const float2 wseg = twiddle_N((bc * ((uint64_t)seg0 & mask)) & mask, N);
    const int64_t tX = s >> 1;
    const int w = (int)(s & 1);
    float2* Fo = F + ((tX * p.M + K) * 2 + w) * p.N_f;
    const int e = __ldg(p.coset_off + c + 1);
    for (int i = __ldg(p.coset_off + c) + tid; i < e; i += FFT_THREADS)
        Fo[__ldg(p.coset_k + i)] = cmul(buf[padi(__ldg(p.coset_m + i))], wseg);
}

// Sum over the pair set of (A_i A_j + B_i B_j + 2 C_i C_j), one block per template.
__device__ __forceinline__ double nn(float4 a, float4 b) {
    return (double)a.x * b.x + (double)a.y * b.y + 2.0 * (double)a.z * b.z;
}

__global__ void norm_kernel(DevParams p, const float4* __restrict__ norm, int64_t t_base,
                            double* __restrict__ Dout) {
    __shared__ double red[32];
    const int64_t t = t_base + blockIdx.x;
    const float4* nt = norm + t * p.Q * p.M;
    const int64_t M = p.M, R = p.R;
    double acc = 0.0;
    for (int64_t idx = threadIdx.x; idx < p.Q * M; idx += blockDim.x) {
        const int Y = (int)(idx / M);
        const int64_t K = idx - Y * M;
        const float4 nY = nt[Y * M + K];
        double s = 0.0;
        for (int X = 0; X < Y; ++X) s += nn(nt[X * M + K], nY);
        for (int64_t Lg = (K - R > 0 ? K - R : 0); Lg < K; ++Lg)
            for (int X = 0; X < p.Q; ++X) {
                if (p.pair_mode == CC_PAIRS_CROSS_ONLY && X == Y) continue;
                s += nn(nt[X * M + Lg], nY);
            }
        if (p.pair_mode == CC_PAIRS_ALL_ORDERED) s = 2.0 * s + nn(nY, nY);
        acc += s;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) Dout[t] = acc;
}

// Stage 3: one thread per (template, bin, chunk of segments); pairs whose later
// segment is K are added at step K, so each unordered pair is visited once.  A chunk
// starts R segments early to see its first segments' partners; the chunk partial
// sums are combined by pair_finalize_kernel.  The segment loop is unrolled twice so
// each thread keeps both segments' spectra loads in flight.
__global__ void __launch_bounds__(PAIR_THREADS)
pair_kernel(DevParams p, const float2* __restrict__ F, int64_t t_base, int64_t chunk_len,
            float* __restrict__ raw) {
    const int64_t t = t_base + blockIdx.z;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.N_f) return;
    const int Q = p.Q;
    const int64_t M = p.M, R = p.R, Nf = p.N_f;
    const int mode = p.pair_mode;
    const int64_t Ka = (int64_t)blockIdx.y * chunk_len;
    const int64_t Kb = Ka + chunk_len < M ? Ka + chunk_len : M;
    const float2* __restrict__ Ft = F + (size_t)t * Q * M * 2 * Nf + k;
    auto Fat = [&](int X, int64_t K, int w) -> float2 {
        return __ldg(Ft + (((size_t)X * M + K) * 2 + w) * Nf);
    };
    auto step = [&](int64_t K, const float2 (&fk)[2][CC_MAX_DET]) -> float {
        float term = 0.f;
        for (int w = 0; w < 2; ++w) {
            float2 winx[CC_MAX_DET];
            float2 win = make_float2(0.f, 0.f);
            for (int X = 0; X < Q; ++X) winx[X] = make_float2(0.f, 0.f);
            for (int64_t Lg = (K - R > 0 ? K - R : 0); Lg < K; ++Lg)
                for (int X = 0; X < Q; ++X) {
                    const float2 f = Fat(X, Lg, w);
                    win = cadd(win, f);
                    winx[X] = cadd(winx[X], f);
                }
            float2 same = make_float2(0.f, 0.f);
            for (int Y = 0; Y < Q; ++Y) {
                const float2 h = cadd(same, mode == CC_PAIRS_CROSS_ONLY ? csub(win, winx[Y]) : win);
                float tY = redot(fk[w][Y], h);
                if (mode == CC_PAIRS_ALL_ORDERED) tY = fmaf(2.f, tY, redot(fk[w][Y], fk[w][Y]));
                term += tY;
                same = cadd(same, fk[w][Y]);
            }
        }
        return term;
    };
    float sum = 0.f, comp = 0.f;
    int64_t K = Ka;
    for (; K + 1 < Kb; K += 2) {
        float2 f0[2][CC_MAX_DET], f1[2][CC_MAX_DET];
        for (int w = 0; w < 2; ++w)
            for (int X = 0; X < Q; ++X) {
                f0[w][X] = Fat(X, K, w);
                f1[w][X] = Fat(X, K + 1, w);
            }
        kahan_add(sum, comp, step(K, f0));
        kahan_add(sum, comp, step(K + 1, f1));
    }
    if (K < Kb) {
        float2 f0[2][CC_MAX_DET];
        for (int w = 0; w < 2; ++w)
            for (int X = 0; X < Q; ++X) f0[w][X] = Fat(X, K, w);
        kahan_add(sum, comp, step(K, f0));
    }
    raw[((size_t)t * gridDim.y + blockIdx.y) * Nf + k] = sum;
}

// Stage 3 for R <= 1: each segment's spectra are read once; the previous segment's stay
// in registers.  Same pair terms and order as pair_kernel.  Four segments per step so
// 4 x 2 x Q loads are in flight per thread.
template <int U, int QT>
__global__ void __launch_bounds__(PAIR_THREADS)
pair_kernel_r1(DevParams p, const float2* __restrict__ F, int64_t t_base, int64_t chunk_len,
               float* __restrict__ raw) {
    const int64_t t = t_base + blockIdx.z;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= p.N_f) return;
    constexpr int Q = QT;
    const int64_t M = p.M, Nf = p.N_f;
    const int mode = p.pair_mode;
    const bool lag = p.R > 0;
    const int64_t Ka = (int64_t)blockIdx.y * chunk_len;
    const int64_t Kb = Ka + chunk_len < M ? Ka + chunk_len : M;
    const float2* __restrict__ Ft = F + (size_t)t * Q * M * 2 * Nf + k;
    auto Fat = [&](int X, int64_t K, int w) -> float2 {
        return __ldg(Ft + (((size_t)X * M + K) * 2 + w) * Nf);
    };
    float2 prev[2][QT];
#pragma unroll
    for (int w = 0; w < 2; ++w)
#pragma unroll
        for (int X = 0; X < QT; ++X)
            prev[w][X] = (lag && Ka > 0) ? Fat(X, Ka - 1, w) : make_float2(0.f, 0.f);
    float sum = 0.f, comp = 0.f;
    for (int64_t K0 = Ka; K0 < Kb; K0 += U) {
        float2 cur[U][2][QT];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int w = 0; w < 2; ++w)
#pragma unroll
                for (int X = 0; X < QT; ++X)
                    cur[u][w][X] = (K0 + u < Kb) ? Fat(X, K0 + u, w) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (K0 + u >= Kb) break;
            float term = 0.f;
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                float2 win = make_float2(0.f, 0.f);
#pragma unroll
                for (int X = 0; X < QT; ++X) win = cadd(win, prev[w][X]);
                float2 same = make_float2(0.f, 0.f);
#pragma unroll
                for (int Y = 0; Y < QT; ++Y) {
                    const float2 h = cadd(same, mode == CC_PAIRS_CROSS_ONLY ? csub(win, prev[w][Y]) : win);
                    float tY = redot(cur[u][w][Y], h);
                    if (mode == CC_PAIRS_ALL_ORDERED) tY = fmaf(2.f, tY, redot(cur[u][w][Y], cur[u][w][Y]));
                    term += tY;
                    same = cadd(same, cur[u][w][Y]);
                }
            }
            kahan_add(sum, comp, term);
#pragma unroll
            for (int w = 0; w < 2; ++w)
#pragma unroll
                for (int X = 0; X < QT; ++X)
                    if (lag) prev[w][X] = cur[u][w][X];
        }
    }
    raw[((size_t)t * gridDim.y + blockIdx.y) * Nf + k] = sum;
}

__global__ void pair_finalize_kernel(const float* __restrict__ raw, const double* __restrict__ Dn,
                                     int64_t N_f, int n_chunks, int64_t t_base, float* __restrict__ rho) {
    const int64_t t = t_base + blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N_f) return;
    float s = 0.f, comp = 0.f;
    for (int c = 0; c < n_chunks; ++c) kahan_add(s, comp, raw[((size_t)t * n_chunks + c) * N_f + k]);
    const double D = Dn[t];
    rho[(size_t)t * N_f + k] = D > 0.0 ? (float)(1.4142135623730951 * (double)s / sqrt(D)) : 0.f;
}

// chunks of segments for the staged pair kernel: enough blocks to fill the GPU, each
// chunk at least 4R + 1 segments long
int64_t pair_chunks(const DevParams& p, int64_t n_t) {
    const int64_t blocks = (int64_t)launch_blocks_for(p.N_f, PAIR_THREADS) * n_t;
    const int64_t want = (8 * 152 + blocks - 1) / (blocks > 0 ? blocks : 1);
    const int64_t maxch = p.M / (4 * p.R + 1) > 0 ? p.M / (4 * p.R + 1) : 1;
    int64_t nch = want < maxch ? want : maxch;
    if (nch < 1) nch = 1;
    if (nch > 65535) nch = 65535;
    return nch;
}

size_t resample_smem_bytes(const DevParams& p, bool window) {
    if (window) return (size_t)resample_window_len(p) * sizeof(float2);
    const int64_t nk = p.N_s / KNOT + 5;
    return (size_t)nk * (sizeof(KnotRec) + sizeof(double));
}

cc_status launch_resample(cc_plan* plan, const cc_template* t_dev, int64_t n_t, void* ab,
                          float* norm, cudaStream_t st, const KnotRec* kn, int64_t nkn, int write_inactive) {
    const DevParams& p = plan->dp;
    // with knot records, the segment's window of x is staged in shared memory when it
    // leaves room for several blocks per SM
    const int use_window = kn && resample_smem_bytes(p, true) <= 96 * 1024;
    const size_t sm = kn ? (use_window ? resample_smem_bytes(p, true) : 0) : resample_smem_bytes(p, false);
    // compile-time half width for the common stencils of the exact interpolator
    const int DT = p.interp == CC_INTERP_EXACT && (p.D == 8 || p.D == 16) ? p.D : 0;
    auto kern = kn ? (DT == 8 ? resample_kernel<8, true> : DT == 16 ? resample_kernel<16, true> : resample_kernel<0, true>)
                   : (DT == 8 ? resample_kernel<8, false> : DT == 16 ? resample_kernel<16, false>
                                                                   : resample_kernel<0, false>);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return cuda_fail(e, "resample smem attribute");
    }
    for (int64_t t0 = 0; t0 < n_t; t0 += MAX_GRID_YZ) {
        const int64_t nt = std::min<int64_t>(MAX_GRID_YZ, n_t - t0);
        dim3 grid((unsigned)p.M, (unsigned)p.Q, (unsigned)nt);
        kern<<<grid, RS_THREADS, sm, st>>>(t_dev, t0, ab, (float4*)norm, kn, nkn, use_window, write_inactive, p);
        count_launch();
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "resample launch");
}

cc_status launch_knots(cc_plan* plan, const cc_template* t_dev, int64_t n_t, KnotRec* kn, cudaStream_t st);

// Knot records of one template's detectors, bytes.
size_t knot_bytes_per_template(const cc_plan* plan) {
    return (size_t)plan->Q * knot_rows(plan) * sizeof(KnotRec);
}

// The complete a_r, b_r and segment norms of n_t templates (the staged stage): FP64 knots
// by the pre-pass for kbatch templates at a time into kn, then the resampling kernel
// with those records, writing zeros where a detector's weights vanish over a segment.
cc_status resample_with_knots(cc_plan* plan, const cc_template* t_dev, int64_t n_t, void* ab, float* norm,
                              cudaStream_t st, KnotRec* kn, int64_t kbatch) {
    const size_t elem = plan->cfg.store == CC_STORE_BF16 ? 4 : 8;
    const size_t ab_t = (size_t)plan->Q * 2 * plan->N_tau * elem;
    const size_t nm_t = (size_t)plan->Q * plan->M * 4;
    const int64_t nkn = knot_rows(plan);
    for (int64_t c0 = 0; c0 < n_t; c0 += kbatch) {
        const int64_t nc = std::min(kbatch, n_t - c0);
        cc_status s = launch_knots(plan, t_dev + c0, nc, kn, st);
        if (s != CC_OK) return s;
        s = launch_resample(plan, t_dev + c0, nc, (char*)ab + ab_t * c0, norm + nm_t * c0, st, kn, nkn, 1);
        if (s != CC_OK) return s;
    }
    return CC_OK;
}

template <int LT>
static const void* segfft_t_ptr() { return (const void*)segfft_kernel_t<LT>; }

cc_status launch_segfft(cc_plan* plan, const void* ab, int64_t n_t, void* F, cudaStream_t st) {
    const DevParams& p = plan->dp;
    // 4096-point cosets of whole segments: the persistent, TMA-staged kernel in spectra mode
    if (plan->segfft_ctr && segfft_tma_supported(plan))
        return launch_segfft_tma(plan, n_t, ab, (float2*)F, plan->segfft_ctr, st);
    const void* kt = p.L == 64 ? segfft_t_ptr<64>() : p.L == 128 ? segfft_t_ptr<128>() : p.L == 256 ? segfft_t_ptr<256>()
                   : p.L == 512 ? segfft_t_ptr<512>() : p.L == 1024 ? segfft_t_ptr<1024>()
                   : p.L == 2048 ? segfft_t_ptr<2048>() : p.L == 4096 ? segfft_t_ptr<4096>() : nullptr;
    if (kt) {
        const size_t smt = (size_t)padded_len(p.L) * sizeof(float2);
        cudaError_t e = cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt);
        if (e != cudaSuccess) return cuda_fail(e, "segment fft smem attribute");
        const int64_t ns = n_t * p.Q * 2;
        for (int64_t s0 = 0; s0 < ns; s0 += MAX_GRID_YZ) {
            const int64_t n = std::min<int64_t>(MAX_GRID_YZ, ns - s0);
            dim3 grid((unsigned)p.C, (unsigned)p.M, (unsigned)n);
            void* args[] = {(void*)&p, (void*)&ab, (void*)&s0, (void*)&F};
            e = cudaLaunchKernel(kt, grid, dim3(FFT_THREADS), args, smt, st);
            count_launch();
            if (e != cudaSuccess) return cuda_fail(e, "segment fft launch");
        }
        return CC_OK;
    }
    const size_t sm = (size_t)2 * p.L * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(segfft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_fail(e, "segment fft smem attribute");
    const int64_t ns = n_t * p.Q * 2;
    for (int64_t s0 = 0; s0 < ns; s0 += MAX_GRID_YZ) {
        const int64_t n = std::min<int64_t>(MAX_GRID_YZ, ns - s0);
        dim3 grid((unsigned)p.C, (unsigned)p.M, (unsigned)n);
        segfft_kernel<<<grid, FFT_THREADS, sm, st>>>(p, ab, s0, (float2*)F);
        count_launch();
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "segment fft launch");
}

cc_status launch_norm_pairs(cc_plan* plan, const void* F, const float* norm, int64_t n_t,
                            double* Dws, float* rawws, float* rho, cudaStream_t st) {
    const DevParams& p = plan->dp;
    const int64_t nch = pair_chunks(p, n_t);
    const int64_t clen = (p.M + nch - 1) / nch;
    const int64_t nchr = (p.M + clen - 1) / clen;
    for (int64_t t0 = 0; t0 < n_t; t0 += MAX_GRID_YZ) {
        const int64_t nt = std::min<int64_t>(MAX_GRID_YZ, n_t - t0);
        norm_kernel<<<(unsigned)nt, 256, 0, st>>>(p, (const float4*)norm, t0, Dws);
        count_launch();
        dim3 grid((unsigned)launch_blocks_for(p.N_f, PAIR_THREADS), (unsigned)nchr, (unsigned)nt);
        if (p.R <= 1 && p.Q == 1)
            pair_kernel_r1<4, 1><<<grid, PAIR_THREADS, 0, st>>>(p, (const float2*)F, t0, clen, rawws);
        else if (p.R <= 1 && p.Q == 2)
            pair_kernel_r1<4, 2><<<grid, PAIR_THREADS, 0, st>>>(p, (const float2*)F, t0, clen, rawws);
        else if (p.R <= 1 && p.Q == 3)
            pair_kernel_r1<4, 3><<<grid, PAIR_THREADS, 0, st>>>(p, (const float2*)F, t0, clen, rawws);
        else if (p.R <= 1)
            pair_kernel_r1<4, 4><<<grid, PAIR_THREADS, 0, st>>>(p, (const float2*)F, t0, clen, rawws);
        else
            pair_kernel<<<grid, PAIR_THREADS, 0, st>>>(p, (const float2*)F, t0, clen, rawws);
        count_launch();
        dim3 g2((unsigned)launch_blocks_for(p.N_f, 256), (unsigned)nt);
        pair_finalize_kernel<<<g2, 256, 0, st>>>(rawws, Dws, p.N_f, (int)nchr, t0, rho);
        count_launch();
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "pair launch");
}

// D per template from the segment norms (t_base.. t_base + n_t - 1 of `norm`)
cc_status launch_norm(cc_plan* plan, const float* norm, int64_t n_t, double* Dws, cudaStream_t st) {
    const DevParams& p = plan->dp;
    for (int64_t t0 = 0; t0 < n_t; t0 += MAX_GRID_YZ) {
        const int64_t nt = std::min<int64_t>(MAX_GRID_YZ, n_t - t0);
        norm_kernel<<<(unsigned)nt, 256, 0, st>>>(p, (const float4*)norm, t0, Dws);
        count_launch();
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "norm launch");
}

// rho = sqrt(2) (sum of n_rows partial rows per template) / sqrt(D)
cc_status launch_pair_finalize(cc_plan* plan, const float* raw, const double* Dws, int n_rows, int64_t n_t,
                               float* rho, cudaStream_t st) {
    const DevParams& p = plan->dp;
    for (int64_t t0 = 0; t0 < n_t; t0 += MAX_GRID_YZ) {
        const int64_t nt = std::min<int64_t>(MAX_GRID_YZ, n_t - t0);
        dim3 g2((unsigned)launch_blocks_for(p.N_f, 256), (unsigned)nt);
        pair_finalize_kernel<<<g2, 256, 0, st>>>(raw, Dws, p.N_f, n_rows, t0, rho);
        count_launch();
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "finalize launch");
}

size_t pair_workspace_bytes(const cc_plan* plan, int64_t n_t) {
    const int64_t nch = pair_chunks(plan->dp, n_t);
    const int64_t clen = (plan->M + nch - 1) / nch;
    const int64_t nchr = (plan->M + clen - 1) / clen;
    return (((size_t)n_t * sizeof(double) + 255) & ~(size_t)255) + (size_t)n_t * nchr * plan->N_f * sizeof(float);
}

cc_status set_inputs(cc_plan* plan, const void* const* x_dev) {
    if (plan->dp.interp == CC_INTERP_LEARNED && !plan->dp.ltaps)
        return fail(CC_ERR_INVALID, "learned interpolation weights not set: call "
                                    "crosscorr_plan_set_learned_interp first");
    if (!x_dev) return fail(CC_ERR_INVALID, "x_dev is null");
    for (int q = 0; q < plan->Q; ++q) {
        if (!x_dev[q]) return fail(CC_ERR_INVALID, "x_dev[" + std::to_string(q) + "] is null");
        if (((uintptr_t)x_dev[q]) & 7) return fail(CC_ERR_INVALID, "x_dev entries must be 8-byte aligned");
        plan->dp.x[q] = (const float2*)x_dev[q];
    }
    return CC_OK;
}

}  // namespace cc

extern "C" {

cc_status crosscorr_resample(cc_plan* plan, const void* const* x_dev, const cc_template* t_dev,
                             int64_t n_t, void* ab_dev, float* norm_dev, void* stream) {
    CC_NVTX_RANGE("crosscorr_resample");
    using namespace cc;
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (n_t < 0) return fail(CC_ERR_INVALID, "n_t must be >= 0");
    if (n_t == 0) return CC_OK;
    if (!t_dev || !ab_dev || !norm_dev) return fail(CC_ERR_INVALID, "null device pointer");
    cc_status s = set_inputs(plan, x_dev);
    if (s != CC_OK) return s;
    // knot records in the plan's workspace, as many templates at a time as it holds (a
    // caller-owned workspace too small for one template's records: knots in each block)
    const size_t krow = knot_bytes_per_template(plan);
    int64_t kbatch;
    if (plan->ws_external) {
        kbatch = std::min<int64_t>(n_t, (int64_t)(plan->ws_bytes / krow));
    } else {
        kbatch = std::max<int64_t>(1, std::min<int64_t>(n_t, (int64_t)(KNOT_WS_BUDGET / krow)));
        if ((s = ensure_workspace(plan, krow * kbatch)) != CC_OK) return s;
    }
    if (kbatch < 1) return launch_resample(plan, t_dev, n_t, ab_dev, norm_dev, (cudaStream_t)stream, nullptr, 0, 0);
    return resample_with_knots(plan, t_dev, n_t, ab_dev, norm_dev, (cudaStream_t)stream, (KnotRec*)plan->ws, kbatch);
}

cc_status crosscorr_segment_fft(cc_plan* plan, const void* ab_dev, int64_t n_t, void* F_dev,
                                void* stream) {
    CC_NVTX_RANGE("crosscorr_segment_fft");
    using namespace cc;
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (n_t < 0) return fail(CC_ERR_INVALID, "n_t must be >= 0");
    if (n_t == 0) return CC_OK;
    if (!ab_dev || !F_dev) return fail(CC_ERR_INVALID, "null device pointer");
    if (plan->M > MAX_GRID_YZ) return fail(CC_ERR_UNSUPPORTED, "more than 65535 segments");
    return launch_segfft(plan, ab_dev, n_t, F_dev, (cudaStream_t)stream);
}

cc_status crosscorr_pair_accumulate(cc_plan* plan, const void* F_dev, const float* norm_dev,
                                    int64_t n_t, float* rho_dev, void* stream) {
    CC_NVTX_RANGE("crosscorr_pair_accumulate");
    using namespace cc;
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (n_t < 0) return fail(CC_ERR_INVALID, "n_t must be >= 0");
    if (n_t == 0) return CC_OK;
    if (!F_dev || !norm_dev || !rho_dev) return fail(CC_ERR_INVALID, "null device pointer");
    cc_status s = ensure_workspace(plan, pair_workspace_bytes(plan, n_t));
    if (s != CC_OK) return s;
    const size_t dbytes = ((size_t)n_t * sizeof(double) + 255) & ~(size_t)255;
    return launch_norm_pairs(plan, F_dev, norm_dev, n_t, (double*)plan->ws,
                             (float*)((char*)plan->ws + dbytes), rho_dev, (cudaStream_t)stream);
}

}  // extern "C"
