// Internal definitions shared by the CUDA translation units of the crosscorr library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "crosscorr.h"

namespace cc {

// Samples between FP64 timing knots.  Between knots the delay d(tau) = tau - t(tau)
// is a cubic through four knots; its error for the Sco X-1 orbit is
// a_p Omega^4 KNOT^4 / 24 * 0.56 ~ 7e-10 s at KNOT = 128.
constexpr int KNOT = 128;
constexpr int MAX_D = 32;
constexpr int MAX_TAPS = 2 * MAX_D + 1;
constexpr int N_BIN_ITER = 4;   // fixed-point steps of the binary delay b = a_p sin(Omega (tau + b - T_asc))
constexpr int N_SSB_ITER = 4;   // fixed-point steps of t = u - Delta(t)
constexpr int N_KEPLER_ITER = 8; // joint fixed-point / Newton steps of the elliptical binary delay
constexpr int MAX_L = 4096;     // largest coset FFT: 256 threads, one radix-16 butterfly each per pass

// Learned interpolator: 8 taps from a 2 -> 64 -> 64 -> 8 tanh network, tabulated at
// LEARNED_NODES offsets u = i / (LEARNED_NODES - 1) and interpolated linearly in u.
// The taps are smooth in u (|d2c/du2| ~ 10), so the table's error is ~1e-6.
constexpr int LEARNED_TAPS = 8;
constexpr int LEARNED_WIDTH = 64;
constexpr int LEARNED_NODES = 1025;
constexpr int LEARNED_TAP_OFFSET = 3;   // first tap at floor(t/dt') - 3

// Timing record of one knot, built from four FP64 knot delays.
struct __align__(16) KnotRec {
    int N;        // floor(d_k / dt)
    float f;      // d_k / dt - N, in [0, 1)
    float psi;    // frac(-f_h d_k - f_r* tau_k), cycles
    float dm1;    // (d_{k-1} - d_k) / dt
    float dp1;    // (d_{k+1} - d_k) / dt
    float dp2;    // (d_{k+2} - d_k) / dt
    float pad0, pad1;
};

// Everything a kernel needs, passed by value.
struct DevParams {
    int Q, D, pair_mode, store;
    int L, C, log2L, nsft;
    int n_ab_step, interp;           // interp: CC_INTERP_EXACT or CC_INTERP_LEARNED
    // floor division of non-negative ints by nsft and n_ab_step: q = (a * m) >> s
    uint32_t nsft_m, ab_m;
    int nsft_s, ab_s;
    int64_t N_t, N_s, M, R, N_tau, N_FFT, N_f;
    int64_t b0;      // (k0 - N_FFT/2) mod N_FFT: FFT bin of output k = 0
    int64_t ab_j0;   // ab_t0 / dt
    double dt, inv_dt, t0, f_h, f_r;
    float f_h_dt, f_r_dt;
    const float2* x[CC_MAX_DET];
    const double* ssb[CC_MAX_DET];
    double eph_t0[CC_MAX_DET], eph_dt[CC_MAX_DET], inv_eph_dt[CC_MAX_DET];
    int64_t n_eph[CC_MAX_DET];
    const float* atab[CC_MAX_DET];
    const float* btab[CC_MAX_DET];
    int64_t n_ab[CC_MAX_DET];
    const float2* sigw[CC_MAX_DET];  // (sigma^2, 1/sigma^2) per T_sft block, (0, 0) in gaps
    int64_t n_sig[CC_MAX_DET];
    const int* lockc[CC_MAX_DET];    // [n_sig + 1] number of locked (sigma > 0) blocks before each block
    const int* coset_off;            // [C+1]
    const int* coset_k;              // [N_f] output index k, grouped by coset
    const int* coset_m;              // [N_f] position in the coset's L-point transform
    const float2* twL;               // exp(-2 pi i j / L), j < L
    const float2* twc;               // [C][N_s]: exp(-2 pi i ((b0 + c) s mod N_FFT) / N_FFT)
    const float2* twk;               // [C4][272]: coset twiddles of the 4096-point kernel's passes (plan.cu)
    int C4;                          // cosets of the 4096-point decomposition (N_FFT / 4096; 0 if N_FFT < 4096)
    int wait_test;                   // crosscorr_plan_set_wait_test: skip each CTA's first bulk copy
    const int* coset4_off;           // [C4+1], and the bin lists of that decomposition
    const int* coset4_k;
    const int* coset4_m;
    unsigned* err;                   // device error word: bit 0 set by a kernel whose bounded wait ran out
    const float* ltaps;              // [LEARNED_NODES][LEARNED_TAPS] learned taps (null until set)
    float ham[MAX_TAPS];             // Hamming window, 2D+1 taps
};

constexpr int FUSED_THREADS = 512;
constexpr int FUSED_WARPS = FUSED_THREADS / 32;
constexpr int MAX_CLUSTER = 8;
constexpr int ACC_SLOTS = 4;   // register pair-sum accumulators per thread (bins per coset <= 2048)
constexpr size_t KNOT_WS_BUDGET = (size_t)8 << 30;   // knot records of one template batch
constexpr int SEGACT_DEPTH = 4;   // ring of per-segment detector-activity flags in the fused kernel

// Shared-memory layout and work split of the fused kernel (byte offsets).
struct FusedLayout {
    int CL;            // CTAs per cluster, sharing each segment
    int S;             // local samples per CTA: its KNOT-sample blocks (block q -> CTA q mod CL)
    int nb;            // max output bins held by one CTA
    int nkseg;         // max knots per segment (incl. the cubic's neighbours)
    int nrec;          // knot records per CTA: two per owned block
    int ring_q;        // detectors kept per ring slot (1: summed; Q: cross-only mode)
    int log2CL;        // CL is a power of two
    int bothw;         // Q <= 2: both weights' transforms buffered, one pair pass per coset
    int regacc;        // one coset per CTA with few bins: pair sums in registers
    int regpair;       // pair sums formed in registers from the last FFT pass (see fused_kernel)
    int mmax;          // largest transform position m of any output bin
    int64_t chunk_len; // segments per chunk
    int n_chunks;
    size_t off_slice, slice_bytes;   // [2][Q][2][S] float2
    size_t off_fft;                  // [weights (2 if bothw)][2 halves][padded L] float2
    size_t off_ring;                 // [slots][ring_q][2][nb] float2; slots = R (summed) or R+1
    size_t off_same;                 // [nb] float2: running detector sum across rounds (Q > 2)
    size_t off_rho;                  // [nb] float, then [nb] float compensation (unless regacc)
    size_t off_dk;                   // [2][Q][nkseg] double
    size_t off_rec;                  // [2][Q][nrec] KnotRec
    size_t off_wpart;                // [2][FUSED_WARPS][Q][4] float
    size_t off_nring;                // [R+1][Q] float4 (rank 0)
    size_t off_bins;                 // [nb] int2 (m, k) and [ncos+1] int starts
    size_t off_flags;                // [SEGACT_DEPTH][CC_MAX_DET] int: detector has weight in a segment
    size_t bytes;
};

}  // namespace cc

// The opaque plan of the C ABI.
struct cc_plan {
    cc_config cfg;
    int Q;
    // plan quantities (host, FP64)
    int64_t N_s, M, R, N_tau, N_FFT, N_f, k0, L, C;
    double T_short, T_coh, dlf, N_FFT0, T_FFT, nu_R, f_r, f_FFT;
    std::vector<int64_t> kbar;
    std::vector<double> freq;
    std::vector<int> coset_off;      // host copy of the coset list offsets [C+1]
    cc::DevParams dp;
    // device allocations owned by the plan
    std::vector<void*> dev_allocs;
    // learned interpolator: device weights (BF16 bits) and tap table, once set
    uint16_t* learned_w = nullptr;
    float* learned_taps = nullptr;
    int search_path = CC_PATH_AUTO;           // crosscorr_plan_set_path
    cc_tuning tuning = {0, 0, 0};             // crosscorr_plan_set_tuning
    int kbar_span4 = 0;                       // largest transform position of a bin, 4096-point cosets
    int* segfft_ctr = nullptr;                // [C4] unit counters of the staged segment FFT (plan-owned)
    bool ws_external = false;                 // ws is caller memory (crosscorr_plan_set_workspace)
    // diagnostic event pairs around fused-kernel launches (crosscorr_plan_set_kernel_timing)
    bool kernel_timing = false;
    std::vector<cudaEvent_t> timing_events;   // [2 * n] start, stop
    size_t timing_used = 0;                   // pairs recorded since the last read
    // detector-frame (demodulation) search: SFT bins and weights, twiddles, bin tables
    void* demod_z = nullptr;                  // [Q][n_blk][nbins] float2
    void* demod_w = nullptr;                  // [Q][n_blk] float4 (a^, b^, locked, 0)
    void* demod_tw = nullptr;                 // [nsft] float2
    void* demod_df = nullptr;                 // [N_f] double: f - f_h of the output bins
    void* demod_kbar = nullptr;               // [N_f] int64
    void* demod_list = nullptr;               // [n_list] int: locked SFTs in time order, 4 l + X
    void* demod_boff = nullptr;               // [n_blk + 1] int: first list entry of each block
    int demod_nlist = 0;
    bool demod_ready = false;
    int demod_form = CC_DEMOD_PAIRS;          // crosscorr_plan_set_demod_form
    int demod_nsft = 0, demod_m_lo = 0, demod_nbins = 0, demod_nblk = 0;
    // workspace (grown on demand by staged/fused paths)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // top-k candidate lists (crosscorr_rho_topk), allocated by its first call
    void* topk_ws = nullptr;
};

namespace cc {

// An NVTX range over one C-ABI call (named in Nsight timelines; without a profiler
// attached the push and pop return at once).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define CC_NVTX_RANGE(name) ::cc::NvtxRange cc_nvtx_range_(name)

// ---------------------------------------------------------------------------
// Host helpers (plan.cu)
// ---------------------------------------------------------------------------
cc_status fail(cc_status s, const std::string& msg);
cc_status cuda_fail(cudaError_t e, const char* what);
cc_status ensure_workspace(cc_plan* p, size_t bytes);
int launch_blocks_for(int64_t n, int threads);
bool fused_layout(const cc_plan* plan, int64_t n_t, FusedLayout* lay);
cc_status launch_fused(cc_plan* plan, const cc_template* t_dev, int64_t n_t, float* rho,
                       const FusedLayout& lay, float* raw, double* dpart, cudaStream_t st,
                       KnotRec* kn_ws = nullptr, int64_t kn_batch = 0);
int64_t knot_rows(const cc_plan* plan);
void count_launch(uint64_t n = 1);
// Event pair for the next timed fused launch (nullptrs when timing is off or fails).
void timing_pair(cc_plan* plan, cudaEvent_t* start, cudaEvent_t* stop);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
// Complex sums and differences as paired FP32 operations (one f32x2 instruction for both
// components, each rounded as the scalar operation): the transforms are bound by
// instruction issue, and a pair takes one issue slot.  a - b is a + (-1) b by one fused
// multiply-add, exact in the product, so it rounds as the subtraction does.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// Re(conj(a) b)
__device__ __forceinline__ float redot(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }
__device__ __forceinline__ float2 mul_negi(float2 a) { return make_float2(a.y, -a.x); }

// Kahan-compensated accumulation.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
    float y = v - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t imax64(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ int floor_div32(int a, int b) {
    int q = a / b;
    return (q * b > a) ? q - 1 : q;
}

// floor(a / b) with the magic pair (m, s) of b (0 <= a < 2^31 exactly; negative a
// through the integer division).
__device__ __forceinline__ int floor_div_magic(int a, int b, uint32_t m, int s) {
    if (a < 0) return floor_div32(a, b);
    return (int)(((uint64_t)(uint32_t)a * m) >> s);
}

// Magic pair for floor division of 0 <= a < 2^31 by 1 <= b < 2^31: with l = ceil(log2 b),
// m = ceil(2^(31 + l) / b) < 2^32 and floor(a / b) = (a m) >> (31 + l) (Granlund and
// Montgomery, "Division by invariant integers using multiplication", Thm. 4.2 with a
// 31-bit dividend).
inline void magic_for(uint32_t b, uint32_t* m, int* s) {
    int l = 0;
    while ((1ull << l) < b) ++l;
    const uint64_t num = (uint64_t)1 << (31 + l);   // l <= 31
    *m = (uint32_t)((num + b - 1) / b);
    *s = 31 + l;
}

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    return (q * b > a) ? q - 1 : q;
}

// Linear interpolation of an FP64 table at time t (end intervals extrapolate);
// inv_dt = 1 / table spacing.
__device__ __forceinline__ double table_lerp(const double* tab, double t0, double inv_dt, int64_t n,
                                             double t) {
    double u = (t - t0) * inv_dt;
    double fi = floor(u);
    int64_t i = (int64_t)fi;
    i = i < 0 ? 0 : (i > n - 2 ? n - 2 : i);
    double f = u - (double)i;
    double v0 = __ldg(tab + i), v1 = __ldg(tab + i + 1);
    return v0 + f * (v1 - v0);
}

// Orbit of one template in the form the timing code uses (times relative to t0).
struct Orbit {
    double a_p, tasc_rel, invP, e;
    double tp_rel;          // periapsis time (elliptical)
    double sinw, cosw, sq;  // sin w, cos w, sqrt(1 - e^2)
};

// sin and cos of an angle in radians through sincospi, whose argument reduction is exact
// (no slow path for large arguments); the rounding of x / pi adds ~1e-16 relative.
__device__ __forceinline__ void sincos_rad(double x, double* s, double* c) {
    sincospi(x * 0.31830988618379067154, s, c);
}

__device__ __forceinline__ Orbit make_orbit(const DevParams& p, const cc_template& T) {
    Orbit o;
    o.a_p = T.a_p;
    o.tasc_rel = T.T_asc - p.t0;
    o.invP = 1.0 / T.P;
    o.e = T.e;
    o.tp_rel = o.tasc_rel;
    o.sinw = 0.0;
    o.cosw = 1.0;
    o.sq = 1.0;
    if (T.e != 0.0) {   // FP64 is slow on this part: circular templates skip these constants
        sincos_rad(T.omega, &o.sinw, &o.cosw);
        o.sq = sqrt(1.0 - T.e * T.e);
        // the ascending node has true anomaly -w: its eccentric and mean anomalies give T_p
        double sh, ch, sEa, cEa;
        sincos_rad(-0.5 * T.omega, &sh, &ch);
        const double Ea = 2.0 * atan2(sqrt(1.0 - T.e) * sh, sqrt(1.0 + T.e) * ch);
        sincos_rad(Ea, &sEa, &cEa);
        o.tp_rel = o.tasc_rel - (Ea - T.e * sEa) * T.P * 0.15915494309189535;
    }
    return o;
}

// d(tau) = tau - t(tau) for detector X and one template (all times relative to t0).
// tau(t) = t_SSB - R(t_SSB)/c, t_SSB = t + Delta_X(t).
// Circular orbit: b = a_p sin(theta0 + Omega b) with theta0 = Omega (tau - T_asc); one
// FP64 sincospi at theta0, then fixed-point steps through the angle-addition formula
// with sin/cos of the small angle Omega b (|Omega b| <= 1.4e-4 rad) from their series
// (remainders below 1e-26); the contraction a_p Omega ~ 1.3e-4 per step leaves
// < 1e-15 s after N_BIN_ITER steps.  Elliptical orbit: b = R(tau + b)/c with E from
// Kepler's equation, one Newton step per fixed-point step from the previous E (the mean
// anomaly moves by Omega db ~ 1e-4 rad per step), N_KEPLER_ITER steps (Newton from
// E = M + e sin M converges quadratically to FP64 precision well within them for e < 0.95).
// SSB part: t = u - Delta(t), u = tau + b, iterated on Delta from Delta(u) (contraction
// |Delta'| <= 1e-4).  Both work on the small quantities b and Delta so d = Delta - b
// keeps FP64 precision.  The binary part depends on the source time only, so a caller
// with several detectors computes it once (knot_binary) and the SSB part per detector
// (knot_ssb); knot_delay is the two together.
__device__ __forceinline__ double knot_binary(const Orbit& o, double tau) {
    double b;
    if (o.e == 0.0) {
        const double x0 = (tau - o.tasc_rel) * o.invP;        // orbital phase in cycles
        double s0, c0;
        sincospi(2.0 * x0, &s0, &c0);
        const double om = 6.283185307179586 * o.invP;         // Omega
        b = o.a_p * s0;
#pragma unroll
        for (int it = 0; it < N_BIN_ITER; ++it) {
            const double dl = om * b, d2 = dl * dl;
            const double sd = dl * (1.0 - d2 * (1.0 / 6.0) * (1.0 - d2 * (1.0 / 20.0)));
            const double cd = 1.0 - d2 * 0.5 * (1.0 - d2 * (1.0 / 12.0));
            b = o.a_p * fma(s0, cd, c0 * sd);
        }
    } else {
        double xm = (tau - o.tp_rel) * o.invP;
        xm -= floor(xm);
        const double M0 = 6.283185307179586 * xm;             // mean anomaly at tau, [0, 2 pi)
        const double om = 6.283185307179586 * o.invP;
        double E = M0 + o.e * sinpi(2.0 * xm), sE, cE;
        sincos_rad(E, &sE, &cE);
        b = 0.0;
#pragma unroll 1
        for (int it = 0; it < N_KEPLER_ITER; ++it) {
            const double M = M0 + om * b;                      // mean anomaly at u = tau + b
            E -= (E - o.e * sE - M) / (1.0 - o.e * cE);
            sincos_rad(E, &sE, &cE);
            b = o.a_p * (o.sinw * (cE - o.e) + o.cosw * o.sq * sE);
        }
    }
    return b;
}

__device__ __forceinline__ double knot_ssb(const DevParams& p, int X, double tau, double b) {
    const double* tab = p.ssb[X];
    const double t0 = p.eph_t0[X], inv = p.inv_eph_dt[X];
    const int64_t n = p.n_eph[X];
    const double u = tau + b;
    double dl = table_lerp(tab, t0, inv, n, u);
#pragma unroll
    for (int it = 0; it < N_SSB_ITER; ++it) dl = table_lerp(tab, t0, inv, n, u - dl);
    return dl - b;
}

__device__ __forceinline__ double knot_delay(const DevParams& p, int X, const Orbit& o, double tau) {
    return knot_ssb(p, X, tau, knot_binary(o, tau));
}

// Knot record from the delays at knots k-1, k, k+1, k+2 (seconds) of a knot at
// source time tau_k.
__device__ __forceinline__ KnotRec make_knot(const DevParams& p, double dm1, double d0,
                                             double dp1, double dp2, double tau_k) {
    KnotRec r;
    double e = d0 * p.inv_dt;
    double fl = floor(e);
    r.N = (int)fl;
    r.f = (float)(e - fl);
    r.dm1 = (float)((dm1 - d0) * p.inv_dt);
    r.dp1 = (float)((dp1 - d0) * p.inv_dt);
    r.dp2 = (float)((dp2 - d0) * p.inv_dt);
    double c = -p.f_h * d0 - p.f_r * tau_k;
    r.psi = (float)(c - floor(c));
    r.pad0 = r.pad1 = 0.f;
    return r;
}

__device__ __forceinline__ KnotRec load_knot(const KnotRec* q) {
    const float4 a = __ldg((const float4*)q), b = __ldg((const float4*)q + 1);
    KnotRec r;
    r.N = __float_as_int(a.x);
    r.f = a.y;
    r.psi = a.z;
    r.dm1 = a.w;
    r.dp1 = b.x;
    r.dp2 = b.y;
    r.pad0 = b.z;
    r.pad1 = b.w;
    return r;
}

// Per-sample timing from the knot record: stencil centre j*, offset delta in
// [-1/2, 1/2) and heterodyne + f_r* phase (cycles, reduced to [-1/2, 1/2)).
struct SampleTiming {
    int jstar;      // sample index of the stencil centre (series fit in 32-bit indices)
    float delta;
    float psi;
};

__device__ __forceinline__ SampleTiming sample_timing(const DevParams& p, const KnotRec& kr,
                                                      int r, int rk) {
    float h = (float)(r - rk) * (1.0f / KNOT);
    float hm1 = h - 1.0f, hm2 = h - 2.0f, hp1 = h + 1.0f;
    float Lm1 = -h * hm1 * hm2 * (1.0f / 6.0f);
    float L1 = -hp1 * h * hm2 * 0.5f;
    float L2 = hp1 * h * hm1 * (1.0f / 6.0f);
    float pp = fmaf(Lm1, kr.dm1, fmaf(L1, kr.dp1, L2 * kr.dp2));
    float v = kr.f + pp;
    float g = 0.5f - v;
    float fl = floorf(g);
    SampleTiming s;
    s.jstar = r - kr.N + (int)fl;
    s.delta = (g - 0.5f) - fl;
    float psi = kr.psi - p.f_h_dt * pp - p.f_r_dt * (float)(r - rk);
    s.psi = psi - rintf(psi);
    return s;
}

// exp(2 pi i psi) for a phase psi in [-1/2, 1/2] cycles (sample_timing reduces it): the
// hardware sine and cosine, whose absolute error on [-pi, pi] is below 4e-7, far inside the
// FP32 parity bar; the full-range sincospif costs several times the instructions in a
// kernel bound by instruction issue.
__device__ __forceinline__ float2 phase_rot(float psi) {
    float s, c;
    __sincosf(6.283185307179586f * psi, &s, &c);
    return make_float2(c, s);
}

// sin(pi r) / (pi r) for |r| <= 1/2 from its Taylor series sum_n (-1)^n (pi r)^2n / (2n+1)!,
// cut after n = 6: the first omitted term is below (pi/2)^14 / 15! = 4.2e-10.
__device__ __forceinline__ float sinc_pi(float r) {
    const float u = 9.86960440108935862f * r * r;   // (pi r)^2
    float s = -1.f / 6227020800.f;                  // -1/13!
    s = fmaf(s, u, 1.f / 39916800.f);               // 1/11!
    s = fmaf(s, u, -1.f / 362880.f);                // -1/9!
    s = fmaf(s, u, 1.f / 5040.f);                   // 1/7!
    s = fmaf(s, u, -1.f / 120.f);                   // -1/5!
    s = fmaf(s, u, 1.f / 6.f);                      // 1/3!
    return fmaf(-s, u, 1.f);                        // 1 - u (1/3! - u/5! + ...)
}

// Windowed-sinc taps on xp[0 .. 2D] (sample j* - D first) at offset delta != 0 (|delta| <=
// 1/2): the sum of xp[n] w_n sinc(delta - (n - D)), with sin(pi (delta - m)) =
// (-1)^m sin(pi delta) and sin(pi delta) / pi = delta sinc_pi(delta).
__device__ __forceinline__ float2 sinc_taps(const DevParams& p, const float2* __restrict__ xp, float delta) {
    const int D = p.D;
    const float s = delta * sinc_pi(delta);                 // sin(pi delta)/pi
    float2 acc = make_float2(0.f, 0.f);
    for (int n = 0; n <= 2 * D; ++n) {
        const float dj = delta - (float)(n - D);              // (t - t_j)/dt
        const float c = p.ham[n] * __fdividef(((n - D) & 1) ? -s : s, dj);
        const float2 xv = xp[n];
        acc.x = fmaf(c, xv.x, acc.x);
        acc.y = fmaf(c, xv.y, acc.y);
    }
    return acc;
}

// sinc_taps for a compile-time half width D, the taps taken in pairs j* -+ k: with
// q = (sin(pi delta)/pi) / (delta^2 - k^2), the coefficients are q (delta -+ k) times the
// signed window (-1)^k w_{D-+k}, so one reciprocal serves two taps.
template <int D>
__device__ __forceinline__ float2 sinc_taps_t(const DevParams& p, const float2* __restrict__ xp, float delta) {
    const float sc = sinc_pi(delta);
    const float s = delta * sc;                              // sin(pi delta)/pi
    const float c0 = p.ham[D] * sc;
    float2 acc = make_float2(c0 * xp[D].x, c0 * xp[D].y);
#pragma unroll
    for (int k = 1; k <= D; ++k) {
        const float q = __fdividef(s, fmaf(delta, delta, -(float)(k * k)));
        const float sg = (k & 1) ? -1.0f : 1.0f;
        const float cm = sg * p.ham[D - k] * q * (delta - (float)k);   // tap j* - k: 1/(delta + k)
        const float cp = sg * p.ham[D + k] * q * (delta + (float)k);   // tap j* + k: 1/(delta - k)
        const float2 xm = xp[D - k], xq = xp[D + k];
        acc.x = fmaf(cm, xm.x, fmaf(cp, xq.x, acc.x));
        acc.y = fmaf(cm, xm.y, fmaf(cp, xq.y, acc.y));
    }
    return acc;
}

// Windowed-sinc interpolation (2D+1 taps) at t/dt = j* + delta of a complex series.
__device__ __forceinline__ float2 interp_sinc(const DevParams& p, const float2* __restrict__ x,
                                              int jstar, float delta) {
    const int N = (int)p.N_t;
    if (delta == 0.0f) {
        return (jstar >= 0 && jstar < N) ? __ldg(x + jstar) : make_float2(0.f, 0.f);
    }
    const int D = p.D;
    const int j0 = jstar - D;
    if (j0 >= 0 && j0 + 2 * D < N) return sinc_taps(p, x + j0, delta);
    const float s = delta * sinc_pi(delta);                 // sin(pi delta)/pi
    float2 acc = make_float2(0.f, 0.f);
    for (int n = 0; n <= 2 * D; ++n) {
        const int j = j0 + n;
        if (j < 0 || j >= N) continue;
        const float dj = delta - (float)(n - D);
        const float c = p.ham[n] * __fdividef(((n - D) & 1) ? -s : s, dj);
        const float2 xv = __ldg(x + j);
        acc.x = fmaf(c, xv.x, acc.x);
        acc.y = fmaf(c, xv.y, acc.y);
    }
    return acc;
}

// Learned taps at offset u in [0, 1) from the tabulated network (linear in u).
__device__ __forceinline__ void learned_coeffs(const DevParams& p, float u, float (&c)[LEARNED_TAPS]) {
    const float fu = u * (float)(LEARNED_NODES - 1);
    int i = (int)fu;
    i = i > LEARNED_NODES - 2 ? LEARNED_NODES - 2 : i;
    const float f = fu - (float)i;
    const float4* tb = (const float4*)(p.ltaps + i * LEARNED_TAPS);
    const float4 a0 = __ldg(tb), a1 = __ldg(tb + 1), n0 = __ldg(tb + 2), n1 = __ldg(tb + 3);
    c[0] = fmaf(f, n0.x - a0.x, a0.x);
    c[1] = fmaf(f, n0.y - a0.y, a0.y);
    c[2] = fmaf(f, n0.z - a0.z, a0.z);
    c[3] = fmaf(f, n0.w - a0.w, a0.w);
    c[4] = fmaf(f, n1.x - a1.x, a1.x);
    c[5] = fmaf(f, n1.y - a1.y, a1.y);
    c[6] = fmaf(f, n1.z - a1.z, a1.z);
    c[7] = fmaf(f, n1.w - a1.w, a1.w);
}

// Learned 8-tap interpolation at t/dt = j* + delta: taps from the tabulated network at
// u = t/dt - floor(t/dt) on x[floor(t/dt) - 3 .. floor(t/dt) + 4].
__device__ __forceinline__ float2 interp_learned(const DevParams& p, const float2* __restrict__ x,
                                                 int jstar, float delta) {
    const int N = (int)p.N_t;
    const bool neg = delta < 0.0f;
    const int j0 = jstar - (neg ? 1 : 0) - LEARNED_TAP_OFFSET;
    float c[LEARNED_TAPS];
    learned_coeffs(p, neg ? delta + 1.0f : delta, c);
    float2 acc = make_float2(0.f, 0.f);
    const bool inside = j0 >= 0 && j0 + LEARNED_TAPS <= N;
#pragma unroll
    for (int n = 0; n < LEARNED_TAPS; ++n) {
        const int j = j0 + n;
        if (!inside && (j < 0 || j >= N)) continue;
        const float2 xv = __ldg(x + j);
        acc.x = fmaf(c[n], xv.x, acc.x);
        acc.y = fmaf(c[n], xv.y, acc.y);
    }
    return acc;
}

// The plan's interpolator (a uniform branch: one plan, one interpolator).
__device__ __forceinline__ float2 interp_sample(const DevParams& p, const float2* __restrict__ x,
                                                int jstar, float delta) {
    return p.interp == CC_INTERP_LEARNED ? interp_learned(p, x, jstar, delta)
                                         : interp_sinc(p, x, jstar, delta);
}

// As interp_sample, reading from a shared-memory copy xs of samples [w0, w0 + nw) of the
// series (zero outside [0, N_t)) when every tap falls inside it, else from x.  DT > 0:
// the windowed sinc's half width D is DT at compile time.
template <int DT = 0>
__device__ __forceinline__ float2 interp_sample_window(const DevParams& p, const float2* __restrict__ x,
                                                       const float2* xs, int w0, int nw, int jstar,
                                                       float delta) {
    if (p.interp == CC_INTERP_LEARNED) {
        const bool neg = delta < 0.0f;
        const int j0 = jstar - (neg ? 1 : 0) - LEARNED_TAP_OFFSET;
        if (j0 < w0 || j0 + LEARNED_TAPS > w0 + nw) return interp_learned(p, x, jstar, delta);
        float c[LEARNED_TAPS];
        learned_coeffs(p, neg ? delta + 1.0f : delta, c);
        const float2* xp = xs + (j0 - w0);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int n = 0; n < LEARNED_TAPS; ++n) {
            acc.x = fmaf(c[n], xp[n].x, acc.x);
            acc.y = fmaf(c[n], xp[n].y, acc.y);
        }
        return acc;
    }
    const int D = DT > 0 ? DT : p.D;
    const int j0 = jstar - D;
    if (j0 < w0 || j0 + 2 * D >= w0 + nw) return interp_sinc(p, x, jstar, delta);
    if (delta == 0.0f) return xs[jstar - w0];
    if constexpr (DT > 0) return sinc_taps_t<DT>(p, xs + (j0 - w0), delta);
    else return sinc_taps(p, xs + (j0 - w0), delta);
}

// Weights at detector time t/dt = j* + delta: alpha = a/sigma^2, beta = b/sigma^2,
// s2 = sigma^2 (all zero in gaps).
struct SampleWeights {
    float alpha, beta, s2;
};

__device__ __forceinline__ SampleWeights sample_weights(const DevParams& p, int X, int jstar,
                                                        float delta) {
    SampleWeights w{0.f, 0.f, 0.f};
    const int q = floor_div_magic(jstar, p.nsft, p.nsft_m, p.nsft_s);
    const int rem = jstar - q * p.nsft;
    const int blk = (rem == 0 && delta < 0.f) ? q - 1 : q;
    if (blk < 0 || blk >= (int)p.n_sig[X]) return w;
    const float2 sw = __ldg(p.sigw[X] + blk);
    const float s2 = sw.x;
    if (!(s2 > 0.f)) return w;
    const int ja = jstar - (int)p.ab_j0;
    const int ia = floor_div_magic(ja, p.n_ab_step, p.ab_m, p.ab_s);
    const int nab = (int)p.n_ab[X];
    const int ic = ia < 0 ? 0 : (ia > nab - 2 ? nab - 2 : ia);
    // the linear interpolant is continuous, so the interval chosen at a node does not matter
    const float fr = ((float)(ja - ic * p.n_ab_step) + delta) / (float)p.n_ab_step;
    const float a0 = __ldg(p.atab[X] + ic), a1 = __ldg(p.atab[X] + ic + 1);
    const float b0 = __ldg(p.btab[X] + ic), b1 = __ldg(p.btab[X] + ic + 1);
    const float a = fmaf(fr, a1 - a0, a0);
    const float b = fmaf(fr, b1 - b0, b0);
    w.alpha = a * sw.y;
    w.beta = b * sw.y;
    w.s2 = s2;
    return w;
}

// exp(-2 pi i j / N) for integer j in [0, N), N a power of two.
__device__ __forceinline__ float2 twiddle_N(uint64_t j, uint64_t N) {
    float s, c;
    sincospif(-2.0f * (float)j / (float)N, &s, &c);
    return make_float2(c, s);
}

// In-place-free Stockham FFT (forward, exp(-2 pi i m s / L)) of L = 2^log2L points in
// shared memory, natural order in and out, radix 4 with one radix-2 pass when log2 L
// is odd.  Input in a, scratch b; returns the buffer holding the result.  Must be
// called by all threads of the block.
__device__ __forceinline__ float2* fft_stockham(float2* a, float2* b, int L, int log2L,
                                                const float2* __restrict__ twL) {
    float2* in = a;
    float2* out = b;
    int Ns = 1;
    const int quarter = L >> 2;
    for (int ps = 0; ps < (log2L >> 1); ++ps) {
        const int stride = L / (Ns * 4);
        for (int j = threadIdx.x; j < quarter; j += blockDim.x) {
            int k = j & (Ns - 1);
            float2 v0 = in[j], v1 = in[j + quarter], v2 = in[j + 2 * quarter], v3 = in[j + 3 * quarter];
            if (Ns > 1) {
                v1 = cmul(v1, __ldg(twL + k * stride));
                v2 = cmul(v2, __ldg(twL + 2 * k * stride));
                v3 = cmul(v3, __ldg(twL + 3 * k * stride));
            }
            float2 a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = mul_negi(csub(v1, v3));
            int idxD = ((j - k) << 2) + k;
            out[idxD] = cadd(a0, a2);
            out[idxD + Ns] = cadd(a1, a3);
            out[idxD + 2 * Ns] = csub(a0, a2);
            out[idxD + 3 * Ns] = csub(a1, a3);
        }
        __syncthreads();
        float2* t = in; in = out; out = t;
        Ns <<= 2;
    }
    if (log2L & 1) {
        const int half = L >> 1;
        const int stride = L / (Ns * 2);
        for (int j = threadIdx.x; j < half; j += blockDim.x) {
            int k = j & (Ns - 1);
            float2 v0 = in[j], v1 = in[j + half];
            if (Ns > 1) v1 = cmul(v1, __ldg(twL + k * stride));
            int idxD = ((j - k) << 1) + k;
            out[idxD] = cadd(v0, v1);
            out[idxD + Ns] = csub(v0, v1);
        }
        __syncthreads();
        float2* t = in; in = out; out = t;
    }
    return in;
}

}  // namespace cc
