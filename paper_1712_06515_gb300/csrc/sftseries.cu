// Heterodyned, downsampled series from SFT bands (Appendix B): per SFT an N'-point
// inverse DFT of the band around k_h with the half-band index shift, the (-1)^j' sign and
// the SFT-start phase exp(-2 pi i f_h (t_K - T_sft/2)) that keeps the SFTs in phase.
// The input preparation of the search (once per dataset, not per template).  N' with
// prime factors 2, 3 and 5 only takes a mixed-radix FFT; any other N' the direct DFT.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"

namespace cc {
namespace {

constexpr int SS_THREADS = 256;
constexpr int SS_WARP_SMEM = 72 * 1024;   // shared-memory budget of a persistent-warp CTA

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

// Mixed-radix transform of N' = product of radices 2, 3, 4, 5 (the 120-day band's
// N' = 360 = 4 x 2 x 3 x 3 x 5): an out-of-place Stockham FFT in shared memory, one pass
// per radix (pass p: butterfly j, k = j mod NS with NS the product of the earlier radices,
// inputs j + r N'/R times W_(NS R)^(k r), outputs at (j - k) R + k + r NS), natural order
// out.  The inverse DFT of Eq. shifted-for-fft is the conjugate of the forward DFT of the
// conjugated band.  N' log N' work instead of the direct DFT's N'^2.
constexpr int SS_MAX_PASSES = 16;
struct Radices {
    int n;
    int r[SS_MAX_PASSES];
    int ns[SS_MAX_PASSES];        // product of the earlier radices
    uint32_t nsm[SS_MAX_PASSES];  // floor(j / ns) = (j nsm) >> nss (magic_for)
    int nss[SS_MAX_PASSES];
    int nb[SS_MAX_PASSES];        // butterflies N' / R
    int tstep[SS_MAX_PASSES];     // twiddle stride N' / (ns R)
};

constexpr float kC3 = 0.866025403784438647f;    // sin(2 pi / 3)
constexpr float kC51 = 0.309016994374947424f;   // cos(2 pi / 5)
constexpr float kC52 = -0.809016994374947424f;  // cos(4 pi / 5)
constexpr float kS51 = 0.951056516295153572f;   // sin(2 pi / 5)
constexpr float kS52 = 0.587785252292473129f;   // sin(4 pi / 5)

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 f2negi(float2 a) { return make_float2(a.y, -a.x); }   // -i a

// forward DFT of radix R in place on v[0 .. R-1] (exp(-2 pi i n k / R))
__device__ __forceinline__ void dft_small(float2 (&v)[5], int R) {
    if (R == 2) {
        const float2 a = v[0];
        v[0] = f2add(a, v[1]);
        v[1] = f2sub(a, v[1]);
    } else if (R == 3) {
        const float2 s = f2add(v[1], v[2]), d = f2sub(v[1], v[2]);
        const float2 t = f2sub(v[0], f2scale(s, 0.5f)), u = f2negi(f2scale(d, kC3));
        v[0] = f2add(v[0], s);
        v[1] = f2add(t, u);
        v[2] = f2sub(t, u);
    } else if (R == 4) {
        const float2 s0 = f2add(v[0], v[2]), d0 = f2sub(v[0], v[2]);
        const float2 s1 = f2add(v[1], v[3]), d1 = f2negi(f2sub(v[1], v[3]));
        v[0] = f2add(s0, s1);
        v[2] = f2sub(s0, s1);
        v[1] = f2add(d0, d1);
        v[3] = f2sub(d0, d1);
    } else {   // R == 5
        const float2 a14 = f2add(v[1], v[4]), d14 = f2sub(v[1], v[4]);
        const float2 a23 = f2add(v[2], v[3]), d23 = f2sub(v[2], v[3]);
        const float2 p1 = make_float2(v[0].x + kC51 * a14.x + kC52 * a23.x, v[0].y + kC51 * a14.y + kC52 * a23.y);
        const float2 p2 = make_float2(v[0].x + kC52 * a14.x + kC51 * a23.x, v[0].y + kC52 * a14.y + kC51 * a23.y);
        const float2 q1 = f2negi(make_float2(kS51 * d14.x + kS52 * d23.x, kS51 * d14.y + kS52 * d23.y));
        const float2 q2 = f2negi(make_float2(kS52 * d14.x - kS51 * d23.x, kS52 * d14.y - kS51 * d23.y));
        v[0] = f2add(v[0], f2add(a14, a23));
        v[1] = f2add(p1, q1);
        v[4] = f2sub(p1, q1);
        v[2] = f2add(p2, q2);
        v[3] = f2sub(p2, q2);
    }
}

// N' above 1536: one T_sft block per CTA (groups = 1), the CTA's barriers ordering the
// passes; twf: forward twiddles exp(-2 pi i e / N').  A gap block writes zeros.
__global__ void __launch_bounds__(SS_THREADS)
sft_fft_kernel(const float2* __restrict__ band, const int64_t* __restrict__ block_sft, int64_t n_blocks,
               int n_prime, double T_sft, double f_h, const float2* __restrict__ twf, Radices rad, int groups,
               float2* __restrict__ x) {
    extern __shared__ __align__(16) float2 sb[];   // per group two buffers of N'
    const int gs = blockDim.x / groups, g = threadIdx.x / gs;
    const int tid = threadIdx.x % gs, nt = gs;
    const int64_t b = (int64_t)blockIdx.x * groups + g;
    const bool have = b < n_blocks;
    const int64_t s = have ? block_sft[b] : -1;
    float2* xo = x + b * (int64_t)n_prime;
    if (have && s < 0)
        for (int j = tid; j < n_prime; j += nt) xo[j] = make_float2(0.f, 0.f);
    const bool work = s >= 0;
    float2* src = sb + (size_t)g * 2 * n_prime;
    float2* dst = src + n_prime;
    if (work) {
        const float2* __restrict__ zs = band + s * (int64_t)n_prime;
        for (int m = tid; m < n_prime; m += nt) {
            const float2 z = __ldg(zs + m);
            src[m] = make_float2(z.x, -z.y);   // conjugated band
        }
    }
    auto sync = [] { __syncthreads(); };
    sync();
    for (int p = 0; p < rad.n; ++p) {
        const int R = rad.r[p], ns = rad.ns[p], nb = n_prime / R, tstep = n_prime / (ns * R);
        const uint32_t nsm = rad.nsm[p];
        const int nss = rad.nss[p];
        for (int j = tid; work && j < nb; j += nt) {
            const int k = j - (int)(((uint64_t)(uint32_t)j * nsm) >> nss) * ns;   // j mod ns
            float2 v[5];
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) v[r] = src[j + r * nb];
            if (ns > 1) {
#pragma unroll
                for (int r = 1; r < 5; ++r)
                    if (r < R) {
                        const float2 w = __ldg(twf + k * r * tstep);
                        v[r] = make_float2(v[r].x * w.x - v[r].y * w.y, v[r].x * w.y + v[r].y * w.x);
                    }
            }
            dft_small(v, R);
            float2* d = dst + (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < 5; ++r)
                if (r < R) d[r * ns] = v[r];
        }
        sync();
        float2* t = src;
        src = dst;
        dst = t;
    }
    if (!work) return;
    // SFT-start phase in FP64, reduced to cycles; output (-1)^j conj(X_j) / T_sft times it
    const double cyc = f_h * ((double)b * T_sft);
    const float c = (float)(cyc - floor(cyc));
    float sn, cs;
    sincospif(2.0f * c, &sn, &cs);
    const float2 rot = make_float2(cs, -sn);
    const float scale = (float)(1.0 / T_sft);
    for (int j = tid; j < n_prime; j += nt) {
        const float sg = (j & 1) ? -scale : scale;
        const float2 a = make_float2(src[j].x * sg, -src[j].y * sg);
        xo[j] = make_float2(fmaf(a.x, rot.x, -a.y * rot.y), fmaf(a.x, rot.y, a.y * rot.x));
    }
}

__device__ __forceinline__ void cp_async8(float2* dst, const float2* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// forward DFT of radix R (compile time) in place on v[0 .. R-1]
template <int R>
__device__ __forceinline__ void dft_r(float2 (&v)[R]) {
    if constexpr (R == 2) {
        const float2 a = v[0];
        v[0] = f2add(a, v[1]);
        v[1] = f2sub(a, v[1]);
    } else if constexpr (R == 3) {
        const float2 s = f2add(v[1], v[2]), d = f2sub(v[1], v[2]);
        const float2 t = f2sub(v[0], f2scale(s, 0.5f)), u = f2negi(f2scale(d, kC3));
        v[0] = f2add(v[0], s);
        v[1] = f2add(t, u);
        v[2] = f2sub(t, u);
    } else if constexpr (R == 4) {
        const float2 s0 = f2add(v[0], v[2]), d0 = f2sub(v[0], v[2]);
        const float2 s1 = f2add(v[1], v[3]), d1 = f2negi(f2sub(v[1], v[3]));
        v[0] = f2add(s0, s1);
        v[2] = f2sub(s0, s1);
        v[1] = f2add(d0, d1);
        v[3] = f2sub(d0, d1);
    } else {
        static_assert(R == 5, "radix 2, 3, 4 or 5");
        const float2 a14 = f2add(v[1], v[4]), d14 = f2sub(v[1], v[4]);
        const float2 a23 = f2add(v[2], v[3]), d23 = f2sub(v[2], v[3]);
        const float2 p1 = make_float2(v[0].x + kC51 * a14.x + kC52 * a23.x, v[0].y + kC51 * a14.y + kC52 * a23.y);
        const float2 p2 = make_float2(v[0].x + kC52 * a14.x + kC51 * a23.x, v[0].y + kC52 * a14.y + kC51 * a23.y);
        const float2 q1 = f2negi(make_float2(kS51 * d14.x + kS52 * d23.x, kS51 * d14.y + kS52 * d23.y));
        const float2 q2 = f2negi(make_float2(kS52 * d14.x - kS51 * d23.x, kS52 * d14.y - kS51 * d23.y));
        v[0] = f2add(v[0], f2add(a14, a23));
        v[1] = f2add(p1, q1);
        v[4] = f2sub(p1, q1);
        v[2] = f2add(p2, q2);
        v[3] = f2sub(p2, q2);
    }
}

// One Stockham pass of radix R over N' points by one warp (lanes stride the butterflies);
// CONJ conjugates the inputs (the first pass, reading the staged band).
template <int R, bool CONJ>
__device__ __forceinline__ void warp_pass_r(const float2* src, float2* dst, const float2* twf, int nb, int tstep,
                                            int ns, uint32_t nsm, int nss, int lane) {
    for (int j = lane; j < nb; j += 32) {
        const int k = ns == 1 ? 0 : j - (int)(((uint64_t)(uint32_t)j * nsm) >> nss) * ns;   // j mod ns
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            v[r] = src[j + r * nb];
            if (CONJ) v[r].y = -v[r].y;
        }
        if (ns > 1) {
            const int tk = k * tstep;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 w = twf[tk * r];
                v[r] = make_float2(v[r].x * w.x - v[r].y * w.y, v[r].x * w.y + v[r].y * w.x);
            }
        }
        dft_r<R>(v);
        float2* d = dst + (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[r * ns] = v[r];
    }
}

template <bool CONJ>
__device__ __forceinline__ void warp_pass(const float2* src, float2* dst, const float2* twf, const Radices& rad,
                                          int p, int lane) {
    const int nb = rad.nb[p], tstep = rad.tstep[p], ns = rad.ns[p], nss = rad.nss[p];
    const uint32_t nsm = rad.nsm[p];
    switch (rad.r[p]) {   // the same for the whole warp
        case 2: warp_pass_r<2, CONJ>(src, dst, twf, nb, tstep, ns, nsm, nss, lane); break;
        case 3: warp_pass_r<3, CONJ>(src, dst, twf, nb, tstep, ns, nsm, nss, lane); break;
        case 4: warp_pass_r<4, CONJ>(src, dst, twf, nb, tstep, ns, nsm, nss, lane); break;
        default: warp_pass_r<5, CONJ>(src, dst, twf, nb, tstep, ns, nsm, nss, lane); break;
    }
}

// N' up to 1536: persistent warps, each taking its next T_sft block from a global counter
// (locked SFTs and gaps fall unevenly on a fixed stride; the counter balances them).  Per
// warp three N'-point shared buffers: the next locked SFT's bins are staged by cp.async
// while the current one runs its passes, so its HBM latency overlaps the transform; the
// forward twiddles exp(-2 pi i e / N') are formed once per CTA (FP64).  Only warp-level
// synchronisation after the one CTA barrier of the twiddle table.
__global__ void __launch_bounds__(SS_THREADS)
sft_fft_warp_kernel(const float2* __restrict__ band, const int64_t* __restrict__ block_sft, int64_t n_blocks,
                    int n_prime, double T_sft, double f_h, Radices rad, unsigned int* __restrict__ next_block,
                    float2* __restrict__ x) {
    extern __shared__ __align__(16) float2 sw[];
    float2* twf = sw;                                  // [N' rounded up to even]
    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* stage = sw + ((n_prime + 1) & ~1) + (size_t)g * 3 * n_prime;
    float2* bufA = stage + n_prime;
    float2* bufB = bufA + n_prime;
    for (int e = threadIdx.x; e < n_prime; e += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)e / (double)n_prime, &sn, &cs);
        twf[e] = make_float2((float)cs, (float)sn);
    }
    __syncthreads();
    auto grab = [&]() -> int64_t {
        unsigned int v = 0;
        if (lane == 0) v = atomicAdd(next_block, 1u);
        return (int64_t)__shfl_sync(0xffffffffu, v, 0);
    };
    int64_t b = grab();
    int64_t s = b < n_blocks ? __ldg(block_sft + b) : -1;
    if (s >= 0) {
        const float2* zs = band + s * (int64_t)n_prime;
        for (int m = lane; m < n_prime; m += 32) cp_async8(stage + m, zs + m);
    }
    cp_async_commit();
    const float scale = (float)(1.0 / T_sft);
    while (b < n_blocks) {
        const int64_t bn = grab();
        const int64_t sn = bn < n_blocks ? __ldg(block_sft + bn) : -1;
        float2* xo = x + b * (int64_t)n_prime;
        if (s >= 0) {
            cp_async_wait_all();
            __syncwarp();
            warp_pass<true>(stage, bufA, twf, rad, 0, lane);
            __syncwarp();                              // the stage is free: every lane has read it
        }
        if (sn >= 0) {
            const float2* zs = band + sn * (int64_t)n_prime;
            for (int m = lane; m < n_prime; m += 32) cp_async8(stage + m, zs + m);
            cp_async_commit();
        }
        if (s >= 0) {
            float2* src = bufA;
            float2* dst = bufB;
            for (int p = 1; p < rad.n; ++p) {
                __syncwarp();
                warp_pass<false>(src, dst, twf, rad, p, lane);
                float2* t = src;
                src = dst;
                dst = t;
            }
            __syncwarp();
            // SFT-start phase in FP64, reduced to cycles; output (-1)^j conj(X_j) / T_sft times it
            const double cyc = f_h * ((double)b * T_sft);
            const float c = (float)(cyc - floor(cyc));
            float sn2, cs;
            sincospif(2.0f * c, &sn2, &cs);
            const float2 rot = make_float2(cs, -sn2);
            for (int j = lane; j < n_prime; j += 32) {
                const float sg = (j & 1) ? -scale : scale;
                const float2 a = make_float2(src[j].x * sg, -src[j].y * sg);
                xo[j] = make_float2(fmaf(a.x, rot.x, -a.y * rot.y), fmaf(a.x, rot.y, a.y * rot.x));
            }
            __syncwarp();                              // bufA / bufB reads done before the next pass 0
        } else {
            for (int j = lane; j < n_prime; j += 32) xo[j] = make_float2(0.f, 0.f);
        }
        s = sn;
        b = bn;
    }
    cp_async_wait_all();
}

// The per-pass constants of a radix order r[0 .. n-1] of N'.
void set_passes(int64_t N, const int* r, int n, Radices* rad) {
    rad->n = n;
    int ns = 1;
    for (int i = 0; i < n; ++i) {
        const int R = r[i];
        rad->ns[i] = ns;
        magic_for((uint32_t)ns, &rad->nsm[i], &rad->nss[i]);
        rad->nb[i] = (int)(N / R);
        rad->tstep[i] = (int)(N / ((int64_t)ns * R));
        rad->r[i] = R;
        ns *= R;
    }
}

// N' as radices 4, 2, 3, 5 (fours first); false if another prime divides it.
bool factor_radices(int64_t n, Radices* rad) {
    int r[SS_MAX_PASSES], k = 0;
    int64_t m = n;
    for (int R : {4, 2, 3, 5}) {
        while (m % R == 0) {
            if (k == SS_MAX_PASSES) return false;
            r[k++] = R;
            m /= R;
        }
    }
    if (m != 1) return false;
    set_passes(n, r, k, rad);
    return true;
}

// Shared-memory wavefronts of one warp access to 8-byte elements at `idx` (32 banks of
// 4 bytes, 128-byte rows): the largest number of distinct rows any bank is asked for.
int warp_wavefronts(const int* idx, int nl) {
    int rows[32][64], cnt[32] = {0};
    int worst = 0;
    for (int l = 0; l < nl; ++l)
        for (int h = 0; h < 2; ++h) {
            const int w = 8 * idx[l] + 4 * h, b = (w / 4) % 32, row = w / 128;
            bool seen = false;
            for (int i = 0; i < cnt[b]; ++i) seen |= rows[b][i] == row;
            if (!seen) {
                rows[b][cnt[b]++] = row;
                worst = std::max(worst, cnt[b]);
            }
        }
    return worst;
}

// Shared-memory wavefronts of the warp kernel's passes in a radix order: the R strided
// reads src[j + r nb], the R writes dst[(j - k) R + k + r NS] and the twiddle reads.
int64_t order_wavefronts(int64_t N, const int* r, int n) {
    int64_t total = 0;
    int ns = 1, idx[32];
    for (int p = 0; p < n; ++p) {
        const int R = r[p], nb = (int)(N / R), tstep = (int)(N / ((int64_t)ns * R));
        for (int j0 = 0; j0 < nb; j0 += 32) {
            const int nl = std::min(32, nb - j0);
            for (int q = 0; q < R; ++q) {
                for (int l = 0; l < nl; ++l) idx[l] = j0 + l + q * nb;
                total += warp_wavefronts(idx, nl);
                for (int l = 0; l < nl; ++l) {
                    const int j = j0 + l, k = j % ns;
                    idx[l] = (j - k) * R + k + q * ns;
                }
                total += warp_wavefronts(idx, nl);
                if (ns > 1 && q > 0) {
                    for (int l = 0; l < nl; ++l) idx[l] = ((j0 + l) % ns) * q * tstep;
                    total += warp_wavefronts(idx, nl);
                }
            }
        }
        ns *= R;
    }
    return total;
}

// The warp kernel's radix order: of every distinct order of the factors, the one with the
// fewest shared-memory wavefronts (early passes write with stride R, and a radix whose
// stride shares no factor with the banks writes without conflicts).
void order_for_banks(int64_t N, Radices* rad) {
    int r[SS_MAX_PASSES], best[SS_MAX_PASSES];
    const int n = rad->n;
    for (int i = 0; i < n; ++i) r[i] = rad->r[i];
    std::sort(r, r + n);
    int64_t best_w = -1;
    do {
        const int64_t w = order_wavefronts(N, r, n);
        if (best_w < 0 || w < best_w) {
            best_w = w;
            std::copy(r, r + n, best);
        }
    } while (std::next_permutation(r, r + n));
    set_passes(N, best, n, rad);
}

}  // namespace
}  // namespace cc

extern "C" cc_status crosscorr_sfts_to_series(const void* band_dev, const int64_t* block_sft_dev, int64_t n_blocks,
                                              int64_t n_prime, double T_sft, double f_h, void* x_dev,
                                              void* stream) {
    CC_NVTX_RANGE("crosscorr_sfts_to_series");
    using namespace cc;
    if (n_blocks < 0 || n_prime < 1 || n_prime > 16384 || !(T_sft > 0) || !std::isfinite(T_sft) ||
        !std::isfinite(f_h))
        return fail(CC_ERR_INVALID, "n_blocks >= 0, 1 <= n_prime <= 16384, T_sft > 0, finite f_h required");
    if (n_blocks == 0) return CC_OK;
    if (!band_dev || !block_sft_dev || !x_dev) return fail(CC_ERR_INVALID, "null device pointer");
    if (n_blocks > 2147483647) return fail(CC_ERR_UNSUPPORTED, "more than 2^31 - 1 blocks");
    Radices rad;
    // the FFT holds two N'-point buffers in shared memory (up to 12800 points)
    const bool fft = n_prime <= 12800 && factor_radices(n_prime, &rad) && rad.n > 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (fft && n_prime <= 1536) {
        // persistent warps: three N'-point buffers per warp plus the CTA's twiddle table,
        // as many warps per CTA (at most 8) as fit in 72 KB; one wave of CTAs
        const size_t per = 3 * sizeof(float2) * n_prime, tw_b = sizeof(float2) * ((n_prime + 1) & ~1);
        const int groups = (int)std::max<int64_t>(1, std::min<int64_t>(SS_THREADS / 32, (SS_WARP_SMEM - tw_b) / per));
        const size_t smem = tw_b + per * groups;
        // the launch shape per (device, N'): the smem attribute and the occupancy query run
        // once, so that repeated calls (and a stream capture of them) only launch
        static std::mutex mu;
        struct Shape {
            int occ, sms;
            Radices rad;
        };
        static std::map<std::pair<int, int64_t>, Shape> shapes;
        int dev = 0, occ = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "sfts_to_series device");
        {
            std::lock_guard<std::mutex> lock(mu);
            auto it = shapes.find({dev, n_prime});
            if (it != shapes.end()) {
                occ = it->second.occ;
                sms = it->second.sms;
                rad = it->second.rad;
            } else {
                order_for_banks(n_prime, &rad);
                // the attribute is the kernel's, shared by every N': set to the largest shape
                // (72 KB, or one group of three 1536-point buffers and the table: 49 KB)
                if ((e = cudaFuncSetAttribute(sft_fft_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              SS_WARP_SMEM)) != cudaSuccess)
                    return cuda_fail(e, "sfts_to_series smem attribute");
                if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sft_fft_warp_kernel, 32 * groups,
                                                                        smem)) != cudaSuccess ||
                    (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                    return cuda_fail(e, "sfts_to_series occupancy");
                shapes[{dev, n_prime}] = Shape{occ, sms, rad};
            }
        }
        const int64_t ctas = std::max<int64_t>(1, std::min<int64_t>((n_blocks + groups - 1) / groups,
                                                                    (int64_t)std::max(1, occ) * sms));
        // the block counter: stream-ordered, zeroed before and freed after the kernel
        unsigned int* ctr = nullptr;
        if ((e = cudaMallocAsync((void**)&ctr, sizeof(unsigned int), st)) != cudaSuccess)
            return cuda_fail(e, "sfts_to_series block counter");
        if ((e = cudaMemsetAsync(ctr, 0, sizeof(unsigned int), st)) != cudaSuccess) {
            cudaFreeAsync(ctr, st);
            return cuda_fail(e, "sfts_to_series block counter");
        }
        sft_fft_warp_kernel<<<(unsigned)ctas, 32 * groups, smem, st>>>((const float2*)band_dev, block_sft_dev,
                                                                       n_blocks, (int)n_prime, T_sft, f_h, rad,
                                                                       ctr, (float2*)x_dev);
        count_launch();
        e = cudaGetLastError();
        cudaFreeAsync(ctr, st);
        return e == cudaSuccess ? CC_OK : cuda_fail(e, "sft_fft_warp_kernel launch");
    }
    // twiddles: exp(+2 pi i j / N') for the direct DFT, exp(-2 pi i j / N') for the FFT
    std::vector<float2> tw(n_prime);
    for (int64_t j = 0; j < n_prime; ++j) {
        const double a = 2.0 * M_PI * (double)j / (double)n_prime;
        tw[j] = make_float2((float)cos(a), (float)(fft ? -sin(a) : sin(a)));
    }
    float2* tw_dev = nullptr;
    e = cudaMallocAsync((void**)&tw_dev, sizeof(float2) * n_prime, st);
    if (e != cudaSuccess) return cuda_fail(e, "sfts_to_series twiddles");
    if ((e = cudaMemcpyAsync(tw_dev, tw.data(), sizeof(float2) * n_prime, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess) {
        cudaFreeAsync(tw_dev, st);
        return cuda_fail(e, "sfts_to_series twiddles");
    }
    if (fft) {
        // one block per CTA, a group of up to 256 threads (a quarter of the widest pass's
        // butterflies), two N'-point buffers
        const size_t smem = 2 * sizeof(float2) * n_prime;
        int rmin = 5;
        for (int i = 0; i < rad.n; ++i) rmin = std::min(rmin, rad.r[i]);
        const int gs = (int)std::min<int64_t>(SS_THREADS, std::max<int64_t>(32, ((n_prime / rmin / 4 + 31) / 32) * 32));
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(sft_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess) {
            cudaFreeAsync(tw_dev, st);
            return cuda_fail(e, "sfts_to_series smem attribute");
        }
        sft_fft_kernel<<<(unsigned)n_blocks, gs, smem, st>>>((const float2*)band_dev, block_sft_dev, n_blocks,
                                                            (int)n_prime, T_sft, f_h, tw_dev, rad, 1,
                                                            (float2*)x_dev);
    } else {
        const size_t smem = sizeof(float2) * n_prime;
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(sft_to_series_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess) {
            cudaFreeAsync(tw_dev, st);
            return cuda_fail(e, "sfts_to_series smem attribute");
        }
        sft_to_series_kernel<<<(unsigned)n_blocks, SS_THREADS, smem, st>>>((const float2*)band_dev, block_sft_dev,
                                                                         (int)n_prime, T_sft, f_h, tw_dev,
                                                                         (float2*)x_dev);
    }
    count_launch();
    e = cudaGetLastError();
    cudaFreeAsync(tw_dev, st);   // stream-ordered: freed after the kernel
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "sft_to_series_kernel launch");
}
