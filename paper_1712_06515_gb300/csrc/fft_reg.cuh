// Register-resident radix-16/8/4/2 DFT kernels and a Stockham pass for L-point FFTs
// (L = 2^n <= 4096) done by 256 threads with one butterfly per thread per pass.
//
// Shared-memory layout: element p of the L-point buffer lives at padi(p) = p + p/16,
// which makes every pass's 8-byte loads and stores bank-conflict free (radix-16
// Stockham writes with stride 16 elements become stride 17).
#pragma once

#include "common.cuh"

namespace cc {

__device__ __forceinline__ int padi(int p) { return p + (p >> 4); }
__host__ __device__ constexpr int padded_len(int L) { return L + L / 16; }

// Padded distance of S consecutive elements when S is a multiple of 16:
// padi(a + r S) = padi(a) + r pstride<S>().
template <int S>
__host__ __device__ constexpr int pstride() {
    static_assert(S % 16 == 0, "padded stride needs a multiple of 16");
    return S + S / 16;
}


// cos(pi/8), sin(pi/8), sqrt(1/2)
constexpr float kC8 = 0.923879532511286756f;
constexpr float kS8 = 0.382683432365089772f;
constexpr float kR2 = 0.707106781186547524f;

__device__ __forceinline__ void dft2(float2& a, float2& b) {
    const float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

// forward 4-point DFT in place, natural order
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 s0 = cadd(a0, a2), d0 = csub(a0, a2), s1 = cadd(a1, a3), d1 = mul_negi(csub(a1, a3));
    a0 = cadd(s0, s1);
    a2 = csub(s0, s1);
    a1 = cadd(d0, d1);
    a3 = csub(d0, d1);
}

// multiplication by exp(-2 pi i e / 16) for the constant exponents of the 4x4 split
template <int E>
__device__ __forceinline__ float2 w16(float2 a) {
    if constexpr (E == 0) return a;
    else if constexpr (E == 1) return cmul(a, make_float2(kC8, -kS8));
    else if constexpr (E == 2) return make_float2(kR2 * (a.x + a.y), kR2 * (a.y - a.x));
    else if constexpr (E == 3) return cmul(a, make_float2(kS8, -kC8));
    else if constexpr (E == 4) return mul_negi(a);
    else if constexpr (E == 6) return make_float2(kR2 * (a.y - a.x), -kR2 * (a.x + a.y));
    else return cmul(a, make_float2(-kC8, kS8));   // E == 9
}

// 16-point DFT: n = 4 n1 + n2, k = k1 + 4 k2; inner 4-point DFTs over n1, twiddles
// W16^(n2 k1), outer 4-point DFTs over n2.  Result in natural order.
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    // v[n2 + 4 k1] = Y[n2][k1]
    v[5] = w16<1>(v[5]);
    v[9] = w16<2>(v[9]);
    v[13] = w16<3>(v[13]);
    v[6] = w16<2>(v[6]);
    v[10] = w16<4>(v[10]);
    v[14] = w16<6>(v[14]);
    v[7] = w16<3>(v[7]);
    v[11] = w16<6>(v[11]);
    v[15] = w16<9>(v[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // v[4 k1 + k2] = X[k1 + 4 k2]: transpose to natural order
    float2 t[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = t[i];
}

// The 16-point DFT of dft16 restricted to its outputs X[0..7], left in v[0..7] (v[8..15]
// hold intermediate values): the outer 4-point DFTs need only their outputs k2 = 0, 1,
// X[k1] = (Y0 + Y2) + (Y1 + Y3) and X[k1 + 4] = (Y0 - Y2) - i (Y1 - Y3).
__device__ __forceinline__ void dft16_lo8(float2 (&v)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    v[5] = w16<1>(v[5]);
    v[9] = w16<2>(v[9]);
    v[13] = w16<3>(v[13]);
    v[6] = w16<2>(v[6]);
    v[10] = w16<4>(v[10]);
    v[14] = w16<6>(v[14]);
    v[7] = w16<3>(v[7]);
    v[11] = w16<6>(v[11]);
    v[15] = w16<9>(v[15]);
    float2 t[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        const float2 a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
        const float2 s0 = cadd(a0, a2), d0 = csub(a0, a2), s1 = cadd(a1, a3), d1 = mul_negi(csub(a1, a3));
        t[k1] = cadd(s0, s1);
        t[k1 + 4] = cadd(d0, d1);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = t[i];
}

// 8-point DFT: n = 4 n1 + n2 (n1 < 2), k = k1 + 2 k2.
__device__ __forceinline__ void dft8(float2 (&v)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft2(v[n2], v[n2 + 4]);
    v[5] = w16<2>(v[5]);   // W8^1
    v[6] = w16<4>(v[6]);   // W8^2
    v[7] = w16<6>(v[7]);   // W8^3
    dft4(v[0], v[1], v[2], v[3]);
    dft4(v[4], v[5], v[6], v[7]);
    float2 t[8];
#pragma unroll
    for (int k1 = 0; k1 < 2; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) t[k1 + 2 * k2] = v[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = t[i];
}

template <int R>
__device__ __forceinline__ void dft_r(float2 (&v)[16]) {
    if constexpr (R == 16) dft16(v);
    else if constexpr (R == 8) dft8(v);
    else if constexpr (R == 4) dft4(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 2) dft2(v[0], v[1]);
}

// v[r] *= W_L^(step r) for r = 1..R-1, from the L-point table: W^step, W^2step,
// W^4step, W^8step are loaded and the rest formed by at most three products.
template <int R>
__device__ __forceinline__ void apply_twiddles(float2 (&v)[16], const float2* __restrict__ twL, int step,
                                               int mask) {
    if constexpr (R == 2) {
        v[1] = cmul(v[1], __ldg(twL + step));
    } else {
        const float2 w1 = __ldg(twL + step);
        const float2 w2 = __ldg(twL + ((2 * step) & mask));
        const float2 w3 = cmul(w2, w1);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        if constexpr (R >= 8) {
            const float2 w4 = __ldg(twL + ((4 * step) & mask));
            v[4] = cmul(v[4], w4);
            v[5] = cmul(v[5], cmul(w4, w1));
            v[6] = cmul(v[6], cmul(w4, w2));
            v[7] = cmul(v[7], cmul(w4, w3));
            if constexpr (R == 16) {
                const float2 w8 = __ldg(twL + ((8 * step) & mask));
                v[8] = cmul(v[8], w8);
#pragma unroll
                for (int r = 9; r < 16; ++r) {
                    const int lo = r - 8;
                    const float2 wl = lo == 1 ? w1 : lo == 2 ? w2 : lo == 3 ? w3 : lo == 4 ? w4
                                    : lo == 5 ? cmul(w4, w1) : lo == 6 ? cmul(w4, w2) : cmul(w4, w3);
                    v[r] = cmul(v[r], cmul(w8, wl));
                }
            }
        }
    }
}

}  // namespace cc

namespace cc {

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

// Compile-time-L versions: constant strides and masks throughout.
template <int R, int L, int NS, typename Sync>
__device__ __forceinline__ void stockham_pass_t(float2* buf, int j, const float2* __restrict__ twL, Sync sync) {
    constexpr int B = L / R;
    float2 v[16];
    const bool act = j < B;
    const int k = j & (NS - 1);
    if (act) {
        if constexpr (B % 16 == 0) {
            const float2* s = buf + padi(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[r * pstride<B>()];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = buf[padi(j + r * B)];
        }
        if constexpr (NS > 1) apply_twiddles<R>(v, twL, k * (L / (NS * R)), L - 1);
        dft_r<R>(v);
    }
    sync();
    if (act) {
        const int idxD = (j - k) * R + k;
        if constexpr (NS % 16 == 0) {
            float2* d = buf + padi(idxD);
#pragma unroll
            for (int r = 0; r < R; ++r) d[r * pstride<NS>()] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) buf[padi(idxD + r * NS)] = v[r];
        }
    }
    sync();
}

template <int L, int NS, typename Sync>
__device__ __forceinline__ void stockham_rest_t(float2* buf, int j, const float2* __restrict__ twL, Sync sync) {
    constexpr int rem = ilog2c(L) - ilog2c(NS);
    if constexpr (rem >= 4) {
        stockham_pass_t<16, L, NS>(buf, j, twL, sync);
        stockham_rest_t<L, NS * 16>(buf, j, twL, sync);
    } else if constexpr (rem == 3) {
        stockham_pass_t<8, L, NS>(buf, j, twL, sync);
    } else if constexpr (rem == 2) {
        stockham_pass_t<4, L, NS>(buf, j, twL, sync);
    } else if constexpr (rem == 1) {
        stockham_pass_t<2, L, NS>(buf, j, twL, sync);
    }
}

}  // namespace cc

namespace cc {

// Radix of the last Stockham pass for an L-point transform whose first pass is radix 16
// and whose later passes are radix 16 while at least four bits remain.
__host__ __device__ constexpr int last_radix(int L) {
    return (ilog2c(L) - 4) % 4 == 0 ? 16 : 1 << ((ilog2c(L) - 4) % 4);
}

// As stockham_rest_t, but the last pass leaves its outputs in registers instead of the
// buffer: thread j < L / last_radix(L) gets outputs j + (L / last_radix(L)) r in v[r],
// r < last_radix(L).  Nothing is written to `buf` by the last pass and no barrier
// follows it; the caller orders any later writes to `buf`.
template <int L, int NS, typename Sync>
__device__ __forceinline__ void stockham_rest_keep_t(float2* buf, int j, const float2* __restrict__ twL,
                                                     Sync sync, float2 (&v)[16]) {
    constexpr int rem = ilog2c(L) - ilog2c(NS);
    static_assert(rem >= 1, "at least one pass after the first");
    if constexpr (rem > 4) {
        stockham_pass_t<16, L, NS>(buf, j, twL, sync);
        stockham_rest_keep_t<L, NS * 16>(buf, j, twL, sync, v);
    } else {
        constexpr int R = 1 << rem;
        static_assert(NS * R == L, "last pass");
        if (j < NS) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = buf[padi(j + r * NS)];
            apply_twiddles<R>(v, twL, j, L - 1);
            dft_r<R>(v);
        }
    }
}

}  // namespace cc

namespace cc {

// One out-of-place Stockham pass (src -> dst, both padded); no barrier inside: the
// caller synchronises before dst is read or src rewritten.
template <int R, int L, int NS>
__device__ __forceinline__ void stockham_pass_oop_t(const float2* src, float2* dst, int j,
                                                    const float2* __restrict__ twL) {
    constexpr int B = L / R;
    if (j < B) {
        float2 v[16];
        const int k = j & (NS - 1);
        const float2* s = src + padi(j);
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[r * pstride<B>()];
        if constexpr (NS > 1) apply_twiddles<R>(v, twL, k * (L / (NS * R)), L - 1);
        dft_r<R>(v);
        float2* d = dst + padi((j - k) * R + k);
#pragma unroll
        for (int r = 0; r < R; ++r) d[r * pstride<NS>()] = v[r];
    }
}

// Passes after the first, out of place (a -> b -> a ...), the last one into registers as
// in stockham_rest_keep_t: one barrier per intermediate pass instead of two.
template <int L, int NS, typename Sync>
__device__ __forceinline__ void stockham_pp_keep_t(float2* a, float2* b, int j, const float2* __restrict__ twL,
                                                   Sync sync, float2 (&v)[16]) {
    constexpr int rem = ilog2c(L) - ilog2c(NS);
    static_assert(rem >= 1, "at least one pass after the first");
    if constexpr (rem > 4) {
        stockham_pass_oop_t<16, L, NS>(a, b, j, twL);
        sync();
        stockham_pp_keep_t<L, NS * 16>(b, a, j, twL, sync, v);
    } else {
        constexpr int R = 1 << rem;
        static_assert(NS * R == L, "last pass");
        if (j < NS) {
            const float2* s = a + padi(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = s[r * pstride<NS>()];
            apply_twiddles<R>(v, twL, j, L - 1);
            dft_r<R>(v);
        }
    }
}

// Number of intermediate passes of stockham_pp_keep_t after a radix-16 first pass; the
// register pass reads the first buffer when it is even.
__host__ __device__ constexpr int pp_intermediate_passes(int L) {
    return (ilog2c(L) - 4 - 1) / 4;
}

}  // namespace cc
