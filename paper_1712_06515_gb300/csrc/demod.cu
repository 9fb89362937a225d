// Detector-frame ("demodulation") CrossCorr: the statistic the resampled method
// replaces (Sec. II: Eqs. fourier-transform-def, normalized-z-bin, total-data-eq,
// geometric-filter, norm-cc, textbook-cc-rho), evaluated at the plan's output
// frequencies on the same data, so the two methods can be compared on one GPU.
//
//   crosscorr_demod_prepare: short Fourier transforms of every locked T_sft block, only
//     the bins a signal in the band can reach (direct DFT with an exact integer twiddle
//     index), normalised to unit variance, and per SFT the filter weights
//     a^ = sqrt(2 T_sft / S) a(t_K), b^ likewise (S = 2 sigma^2 dt);
//   crosscorr_demod_search: per template an FP64 pass gives, per locked SFT (a list in
//     time order built by the prepare call), the signal's bin position and phase as
//     linear functions of the output bin; one thread per (template, output bin) then
//     walks the SFTs in time order, forms
//     y_K = sum_m (-1)^m sinc(kappa_Km) z_Km exp(-i Phi_K) (= Xi_K z_K exp(-i Phi_K)) and
//     sums Gamma_KL 2 Re(conj(y_K) y_L) over every earlier SFT L within T_max, with the
//     normalisation sum (Xi_K Xi_L Gamma_KL)^2 alongside; rho = raw / sqrt(2 den).  Two
//     forms of that sum: the method's pair loop (demod_pair_kernel, one term per pair,
//     each unordered pair once) and the separable form (demod_sep_kernel: Gamma_KL is a
//     sum of products of a K factor and an L factor, so running sums over the partners
//     give the same value in O(1) per SFT).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace cc {
cc_status set_inputs(cc_plan* plan, const void* const* x_dev);

namespace {

constexpr int SFT_THREADS = 256;
constexpr int DM_MAX_SFT_SAMPLES = 16384;   // T_sft / dt staged in shared memory
constexpr size_t DM_RING_BUDGET = 160 * 1024;
constexpr size_t DM_SEP_RING = 40 * 1024;   // separable form: block-sum ring per CTA (R_s <= 10)

struct DemodTiming {   // per (template, locked SFT): 32 bytes
    float A0, A1;       // signal bin position x = A0 + df A1 (df = f - f_h of the output bin)
    float C0, C1;       // heterodyned phase (cycles) = C0 + kbar C1 with kbar = 128 kh + kl:
    float C128, pad0;   //   C0 + kh C128 + kl C1 (mod 1); pad0, pad1: the SFT's a^, b^
    float pad1, pad2;   //   divided by sqrt(10); pad2: its list key 4 l + X (int bits)
};

// DFT bins m_lo .. m_lo + nbins - 1 of one T_sft block of detector X, normalised to unit
// variance, each times (-1)^m: the two-bin interpolation's alternating sign
// (-1)^m0 (s0 z_m0 - s1 z_(m0+1)) is then s0 z'_m0 + s1 z'_(m0+1).  Zero for gaps.  Also the
// block's filter weights (a^, b^, locked).
__global__ void __launch_bounds__(SFT_THREADS)
sft_kernel(DevParams p, int nsft, int m_lo, int nbins, int n_blk, const float2* __restrict__ tw,
           float2* __restrict__ z, float4* __restrict__ wts) {
    extern __shared__ __align__(16) float2 xs[];
    const int l = blockIdx.x, X = blockIdx.y;
    float2* zo = z + ((size_t)X * n_blk + l) * nbins;
    const float2 sw = (l < (int)p.n_sig[X]) ? __ldg(p.sigw[X] + l) : make_float2(0.f, 0.f);
    const bool locked = sw.x > 0.f;
    if (threadIdx.x == 0) {
        float ah = 0.f, bh = 0.f;
        if (locked) {
            // a, b at the mid-time (linear in the table, end intervals extrapolated)
            const double tm = (double)l * nsft + 0.5 * nsft;
            const double fr = (tm - (double)p.ab_j0) / (double)p.n_ab_step;
            int64_t i = (int64_t)floor(fr);
            const int64_t nab = p.n_ab[X];
            i = i < 0 ? 0 : (i > nab - 2 ? nab - 2 : i);
            const double f = fr - (double)i;
            const double a = __ldg(p.atab[X] + i) + f * (__ldg(p.atab[X] + i + 1) - __ldg(p.atab[X] + i));
            const double b = __ldg(p.btab[X] + i) + f * (__ldg(p.btab[X] + i + 1) - __ldg(p.btab[X] + i));
            const double sc = sqrt((double)nsft * (double)sw.y);   // sqrt(2 T_sft / S) = sqrt(nsft / sigma^2)
            ah = (float)(sc * a);
            bh = (float)(sc * b);
        }
        wts[(size_t)X * n_blk + l] = make_float4(ah, bh, locked ? 1.f : 0.f, 0.f);
    }
    if (!locked) {
        for (int i = threadIdx.x; i < nbins; i += blockDim.x) zo[i] = make_float2(0.f, 0.f);
        return;
    }
    const float2* __restrict__ x = p.x[X] + (size_t)l * nsft;
    for (int j = threadIdx.x; j < nsft; j += blockDim.x) xs[j] = __ldg(x + j);
    __syncthreads();
    const float norm = sqrtf(sw.y / (float)nsft);   // dt sqrt(2 / (T_sft S)) = 1 / (sigma sqrt(nsft))
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
        const int m = m_lo + i;
        const int step = ((m % nsft) + nsft) % nsft;     // exp(-2 pi i j m / nsft) = tw[(j m) mod nsft]
        int idx = 0;
        float2 acc = make_float2(0.f, 0.f);
        for (int j = 0; j < nsft; ++j) {
            const float2 w = tw[idx];
            const float2 v = xs[j];
            acc.x = fmaf(v.x, w.x, fmaf(-v.y, w.y, acc.x));
            acc.y = fmaf(v.x, w.y, fmaf(v.y, w.x, acc.y));
            idx += step;
            idx -= idx >= nsft ? nsft : 0;
        }
        const float sn = (m & 1) ? -norm : norm;         // stored times (-1)^m (see below)
        zo[i] = make_float2(acc.x * sn, acc.y * sn);
    }
}

// Per (template, detector, SFT block): the signal's heterodyned bin position and phase as
// functions of the output bin, in FP64 reduced to FP32 pieces.
__device__ DemodTiming demod_timing(const DevParams& p, const cc_template& T, int nsft, int l, int X, double df0,
                                    double dK) {
    const double tmid = ((double)l * nsft + 0.5 * nsft) * p.dt;   // relative to t0
    // Delta_X(t) and its slope (linear interpolation of the table)
    const double u = (tmid - p.eph_t0[X]) * p.inv_eph_dt[X];
    int64_t i = (int64_t)floor(u);
    const int64_t n = p.n_eph[X];
    i = i < 0 ? 0 : (i > n - 2 ? n - 2 : i);
    const double d0 = __ldg(p.ssb[X] + i), d1 = __ldg(p.ssb[X] + i + 1);
    const double dl = d0 + (u - (double)i) * (d1 - d0);
    const double ddl = (d1 - d0) * p.inv_eph_dt[X];
    // binary delay R/c at t_SSB and its rate (Eqs. t-ssb-equation, tau-equation,
    // Kepler-equation), dtau/dt = (1 + Delta') (1 - dR/du / c)
    const Orbit o = make_orbit(p, T);
    const double u_ssb = tmid + dl, om = 6.283185307179586 * o.invP;
    double R, dR;
    if (o.e == 0.0) {
        double s, c;
        sincospi(2.0 * ((u_ssb - o.tasc_rel) * o.invP), &s, &c);
        R = o.a_p * s;
        dR = o.a_p * om * c;
    } else {
        double xm = (u_ssb - o.tp_rel) * o.invP;
        xm -= floor(xm);
        const double M = 6.283185307179586 * xm;
        double E = M + o.e * sinpi(2.0 * xm), sE, cE;
        sincos_rad(E, &sE, &cE);
        for (int it = 0; it < N_KEPLER_ITER; ++it) {
            E -= (E - o.e * sE - M) / (1.0 - o.e * cE);
            sincos_rad(E, &sE, &cE);
        }
        R = o.a_p * (o.sinw * (cE - o.e) + o.cosw * o.sq * sE);
        dR = o.a_p * (-o.sinw * sE + o.cosw * o.sq * cE) * om / (1.0 - o.e * cE);
    }
    const double d = dl - R;                                           // tau - t
    const double dtau = (1.0 + ddl) * (1.0 - dR);
    const double Tsft = nsft * p.dt;
    DemodTiming r;
    // x = (f (dtau - 1) + df) T_sft with f = f_h + df
    r.A0 = (float)(p.f_h * (dtau - 1.0) * Tsft);
    r.A1 = (float)(dtau * Tsft);
    // phase f tau - f_h t = f_h d + df (t + d), df = df0 + kbar dK
    const double tau = tmid + d;
    const double c0 = p.f_h * d + df0 * tau;
    const double c1 = dK * tau, c128 = 128.0 * dK * tau;
    r.C0 = (float)(c0 - floor(c0));
    r.C1 = (float)(c1 - floor(c1));
    r.C128 = (float)(c128 - floor(c128));
    r.pad0 = r.pad1 = r.pad2 = 0.f;
    return r;
}

// The search kernels' records: one per locked SFT of the time-ordered list, the timing of
// demod_timing with the SFT's filter weights (divided by sqrt(10)) and list key (4 l + X) in
// the spare words; two padding records (no bins) follow the list.
__global__ void demod_timing_list_kernel(DevParams p, const cc_template* __restrict__ tm, int nsft, int n_blk,
                                         double df0, double dK, const int* __restrict__ list, int n_list,
                                         const float4* __restrict__ wts, DemodTiming* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t t = blockIdx.y;
    if (i >= n_list + 2) return;
    DemodTiming r;
    if (i >= n_list) {                                 // padding: no bins (x far below the band)
        r.A0 = -1.0e9f;
        r.A1 = r.C0 = r.C1 = r.C128 = r.pad0 = r.pad1 = 0.f;
        r.pad2 = __int_as_float(__ldg(list + n_list - 1));
    } else {
        const int key = __ldg(list + i);
        const int l = key >> 2, X = key & 3;
        r = demod_timing(p, tm[t], nsft, l, X, df0, dK);
        const float4 wk = __ldg(wts + (size_t)X * n_blk + l);
        r.pad0 = wk.x * 0.316227766016837933f;         // a^ / sqrt(10)
        r.pad1 = wk.y * 0.316227766016837933f;
        r.pad2 = __int_as_float(key);
    }
    out[(size_t)t * (n_list + 2) + i] = r;
}

// The same statistic in separable form.  The geometric filter Gamma_KL = (a^_K a^_L +
// b^_K b^_L) / 10 splits into a factor of K times one of L, so the pair sum of SFT K over
// its partners L is 2 Re(conj(y_K) (a^_K SA + b^_K SB)) / 10 with SA = sum_L a^_L y_L and
// SB = sum_L b^_L y_L, and the normalisation term Xi_K^2 (a^_K^2 UAA + 2 a^_K b^_K UAB +
// b^_K^2 UBB) / 100 with UAA = sum_L Xi_L^2 a^_L^2, UAB = sum_L Xi_L^2 a^_L b^_L,
// UBB = sum_L Xi_L^2 b^_L^2: O(1) per SFT instead of one term per partner.  The partners
// of (block l, detector X) are every detector of blocks l - R_s .. l - 1 (window sums W)
// and the earlier detectors of block l (running sums P).  W moves by adding the finished
// block's sums s_l and subtracting s_(l - R_s), and is recomputed exactly every few blocks
// so that rounding cannot drift.  s_(l - R_s) comes from a per-thread ring of block sums in
// shared memory when R_s is small (RING), otherwise it is recomputed from the SFT bins.
// Results equal the per-pair loop's up to FP32 rounding.
struct SepSums {
    float ayx, ayy, byx, byy, uaa, uab, ubb;
};

__device__ __forceinline__ void sep_zero(SepSums& a) { a = SepSums{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}; }

__device__ __forceinline__ void sep_axpy(SepSums& a, const SepSums& b, float sg) {
    a.ayx = fmaf(sg, b.ayx, a.ayx);
    a.ayy = fmaf(sg, b.ayy, a.ayy);
    a.byx = fmaf(sg, b.byx, a.byx);
    a.byy = fmaf(sg, b.byy, a.byy);
    a.uaa = fmaf(sg, b.uaa, a.uaa);
    a.uab = fmaf(sg, b.uab, a.uab);
    a.ubb = fmaf(sg, b.ubb, a.ubb);
}

// SFT (X, l)'s contribution (a^ y, b^ y, Xi^2 a^^2, Xi^2 a^ b^, Xi^2 b^^2) to the sums
__device__ __forceinline__ void sep_add_sft(SepSums& a, float2 y, float xi2, float4 wk) {
    const float xa = xi2 * wk.x, xb = xi2 * wk.y;
    a.ayx = fmaf(wk.x, y.x, a.ayx);
    a.ayy = fmaf(wk.x, y.y, a.ayy);
    a.byx = fmaf(wk.y, y.x, a.byx);
    a.byy = fmaf(wk.y, y.y, a.byy);
    a.uaa = fmaf(xa, wk.x, a.uaa);
    a.uab = fmaf(xa, wk.y, a.uab);
    a.ubb = fmaf(xb, wk.y, a.ubb);
}

// One SFT's inputs for the separable kernel, fetched ahead of its arithmetic: kappa =
// floor(x) - x of the signal bin position, the heterodyne phase in cycles reduced to
// [-1/2, 1/2], and the two stored bins floor(x), floor(x) + 1 (zero when out of the band).
struct SftIn {
    float k0, cyc;
    float2 z0, z1;
};

// The demodulated bin y (the two-bin sinc interpolation of the pair kernel, rotated by the
// heterodyne phase) and the interpolation weight Xi^2.  The two sinc weights
// s0 = sin(pi kappa) / (pi kappa), s1 = -sin(pi kappa) / (pi (kappa + 1)) take the series
// at whichever of kappa, kappa + 1 lies within 1/2 of zero and one quotient for the other
// (its denominator at least 1/2 in size).  The rotation takes the phase in [-1/2, 1/2)
// cycles to the fast sine/cosine, whose absolute error there (2^-21.4) is far below the
// statistic's FP32 rounding.
__device__ __forceinline__ float2 sft_y(const SftIn& q, float& xi2) {
    const bool near0 = q.k0 >= -0.5f;                // kappa in [-1/2, 0]: series at kappa
    const float r = near0 ? q.k0 : q.k0 + 1.f;
    const float far = near0 ? q.k0 + 1.f : q.k0;
    const float sv = sinc_pi(r);
    const float other = -__fdividef(r * sv, far);
    const float s0 = near0 ? sv : other, s1 = near0 ? other : sv;
    xi2 = s0 * s0 + s1 * s1;
    const float2 u = make_float2(fmaf(s0, q.z0.x, s1 * q.z1.x), fmaf(s0, q.z0.y, s1 * q.z1.y));
    float sn, cs;
    __sincosf(6.28318530717958648f * q.cyc, &sn, &cs);
    return make_float2(fmaf(u.x, cs, u.y * sn), fmaf(u.y, cs, -u.x * sn));
}

// One record of the separable kernel's list: timing, weights and key of SFT i.
struct SepRec {
    float4 t0;   // A0, A1, C0, C1
    float4 t1;   // C128, a^, b^, key (int bits: 4 l + X)
};

__device__ __forceinline__ SepRec load_rec(const DemodTiming* __restrict__ r) {
    const float4* q = reinterpret_cast<const float4*>(r);
    return SepRec{__ldg(q), __ldg(q + 1)};
}

__device__ __forceinline__ void rec_fetch(SftIn& q, const SepRec& r, float df, float kh, float kl, int m_lo,
                                          int nbins, int n_blk, const float2* __restrict__ z) {
    const int key = __float_as_int(r.t1.w);
    const float x = fmaf(df, r.t0.y, r.t0.x);
    const float fm = floorf(x);
    q.k0 = fm - x;
    const int idx = (int)fm - m_lo;
    const float cyc = fmaf(kl, r.t0.w, fmaf(kh, r.t1.x, r.t0.z));
    q.cyc = cyc - rintf(cyc);
    q.z0 = q.z1 = make_float2(0.f, 0.f);
    if (idx >= 0 && idx + 1 < nbins) {
        const float2* zr = z + ((size_t)(key & 3) * n_blk + (key >> 2)) * nbins + idx;
        q.z0 = __ldg(zr);
        q.z1 = __ldg(zr + 1);
    }
}

// One thread per (template, output bin) walks the list of locked SFTs in time order (gaps
// never enter the loop).  The SFT records of one template are shared by its CTAs; their
// filter weights come scaled by 1/sqrt(10), so Gamma_KL = a^'_K a^'_L + b^'_K b^'_L and the
// factors 1/10 and 1/100 drop out (the pair sum is then half the statistic's raw sum).
// V holds the sums over SFT K's partners so far (window W plus the current block); block
// sums go to the window when the block index changes: one step adds s_l and subtracts
// s_(l - R_s); a jump over empty blocks, and every 4 (R_s + 1) steps, sums the window
// exactly.  The record list carries two padding records (no bins) past its end so that
// the pipeline's loads need no guards.
template <bool RING>
__global__ void __launch_bounds__(128) demod_sep_kernel(DevParams p, int m_lo, int nbins, int n_blk, int Rs, int refresh,
                                 const float2* __restrict__ z, const DemodTiming* __restrict__ recs, int n_list,
                                 const int* __restrict__ boff, const double* __restrict__ dfreq,
                                 const int64_t* __restrict__ kbar, int64_t t_base, float* __restrict__ rho) {
    extern __shared__ __align__(16) float sring[];     // RING: [R_s + 1][7][nthr] block sums, thread-private
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int64_t t = t_base + blockIdx.y;
    const int k = blockIdx.x * nthr + tid;
    const bool act = k < (int)p.N_f;
    const DemodTiming* rt = recs + (size_t)(t - t_base) * (n_list + 2);
    if (n_list == 0) {                                 // no locked SFT
        if (act) rho[(size_t)t * p.N_f + k] = 0.f;
        return;
    }
    if (RING)
        for (int j = 0; j < (Rs + 1) * 7; ++j) sring[(size_t)j * nthr + tid] = 0.f;
    // threads past the last bin compute bin 0's statistic and store nothing
    const float df = (float)__ldg(dfreq + (act ? k : 0));
    const int64_t kb = __ldg(kbar + (act ? k : 0));
    const float kh = (float)(kb >> 7), kl = (float)(kb & 127);
    auto ring_get = [&](int slot) {
        const float* r = sring + (size_t)slot * 7 * nthr + tid;
        return SepSums{r[0], r[nthr], r[2 * nthr], r[3 * nthr], r[4 * nthr], r[5 * nthr], r[6 * nthr]};
    };
    auto ring_put = [&](int slot, const SepSums& v) {
        float* r = sring + (size_t)slot * 7 * nthr + tid;
        r[0] = v.ayx;
        r[nthr] = v.ayy;
        r[2 * nthr] = v.byx;
        r[3 * nthr] = v.byy;
        r[4 * nthr] = v.uaa;
        r[5 * nthr] = v.uab;
        r[6 * nthr] = v.ubb;
    };
    // block j's sums from its SFT bins (no ring)
    auto block_sums = [&](int j, SepSums& sj) {
        sep_zero(sj);
        const int e = __ldg(boff + j + 1);
        for (int i = __ldg(boff + j); i < e; ++i) {
            const SepRec r = load_rec(rt + i);
            SftIn q;
            rec_fetch(q, r, df, kh, kl, m_lo, nbins, n_blk, z);
            float xi2;
            const float2 y = sft_y(q, xi2);
            sep_add_sft(sj, y, xi2, make_float4(r.t1.y, r.t1.z, 1.f, 0.f));
        }
    };
    float raw = 0.f, rawc = 0.f, den = 0.f, denc = 0.f;
    SepSums W, V;
    sep_zero(W);
    sep_zero(V);
    int steps = 0;
    int lcur = 0, scur = 0;                            // block lcur and its ring slot lcur mod (R_s + 1)
    // the pair and normalisation terms go to plain FP32 partial sums that join the
    // compensated totals at most every 64 SFTs (at a block change)
    float raw_p = 0.f, den_p = 0.f;
    int nacc = 0;
    // SFT i: Rc its record, Fc its fetched inputs; Rn the record of SFT i + 1, Fn receives
    // SFT i + 1's inputs.  The bins of SFT i + 1 and the record of SFT i + 2 (into Rc once
    // read) load while SFT i is summed; two calls per iteration with the roles swapped keep
    // the pipeline in place without register copies.
    auto step = [&](SepRec& Rc, SftIn& Fc, const SepRec& Rn, SftIn& Fn, int i) {
        rec_fetch(Fn, Rn, df, kh, kl, m_lo, nbins, n_blk, z);
        const float4 wk = make_float4(Rc.t1.y, Rc.t1.z, 1.f, 0.f);
        const int l = __float_as_int(Rc.t1.w) >> 2;
        Rc = load_rec(rt + i + 2);
        if (l != lcur) {                               // block lcur is complete: the window of block l
            if (Rs > 0) {
                if (RING) {
                    const bool step1 = l == lcur + 1 && ++steps < refresh;
                    SepSums Pb = V;                    // block lcur's sums
                    sep_axpy(Pb, W, -1.f);
                    ring_put(scur, Pb);
                    if (step1) {
                        scur = scur == Rs ? 0 : scur + 1;       // slot of l: s_(l - R_s - 1) = s_(lcur - R_s)
                        const SepSums old = ring_get(scur);
                        W = V;
                        sep_axpy(W, old, -1.f);
                    } else {
                        const SepSums zero{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        const int nz = min(l - lcur - 1, Rs + 1);   // empty blocks lcur + 1 .. l - 1
                        for (int j = 1; j <= nz; ++j) {
                            scur = scur == Rs ? 0 : scur + 1;
                            ring_put(scur, zero);
                        }
                        scur = l % (Rs + 1);
                        sep_zero(W);
                        for (int j = 0; j <= Rs; ++j)
                            if (j != scur) sep_axpy(W, ring_get(j), 1.f);
                        steps = 0;
                    }
                } else if (l - lcur > Rs) {            // every block of the new window is empty
                    sep_zero(W);
                    steps = 0;
                } else if (++steps < refresh) {        // blocks lcur - R_s .. l - R_s - 1 leave
                    W = V;
                    for (int j = max(0, lcur - Rs); j < l - Rs; ++j) {
                        SepSums old;
                        block_sums(j, old);
                        sep_axpy(W, old, -1.f);
                    }
                } else {
                    SepSums Wn = V;                    // blocks l - R_s .. lcur (those after are empty)
                    sep_axpy(Wn, W, -1.f);
                    for (int j = max(0, l - Rs); j < lcur; ++j) {
                        SepSums sj;
                        block_sums(j, sj);
                        sep_axpy(Wn, sj, 1.f);
                    }
                    W = Wn;
                    steps = 0;
                }
            }
            V = W;
            lcur = l;
            if (steps == 0 || nacc >= 64) {
                kahan_add(raw, rawc, raw_p);
                kahan_add(den, denc, den_p);
                raw_p = den_p = 0.f;
                nacc = 0;
            }
        }
        float xi2;
        const float2 y = sft_y(Fc, xi2);
        const float gx = fmaf(wk.x, V.ayx, wk.y * V.byx), gy = fmaf(wk.x, V.ayy, wk.y * V.byy);
        raw_p = fmaf(y.x, gx, fmaf(y.y, gy, raw_p));                 // Re(conj(y) g)
        const float nq = fmaf(wk.x * wk.x, V.uaa, fmaf(2.f * wk.x * wk.y, V.uab, wk.y * wk.y * V.ubb));
        den_p = fmaf(xi2, nq, den_p);
        ++nacc;
        sep_add_sft(V, y, xi2, wk);
    };
    SepRec ra = load_rec(rt);
    SepRec rb = load_rec(rt + 1);
    SftIn fa, fb;
    rec_fetch(fa, ra, df, kh, kl, m_lo, nbins, n_blk, z);
    lcur = __float_as_int(ra.t1.w) >> 2;
    scur = lcur % (Rs + 1);
    int i = 0;
    for (; i + 1 < n_list; i += 2) {
        step(ra, fa, rb, fb, i);
        step(rb, fb, ra, fa, i + 1);
    }
    if (i < n_list) step(ra, fa, rb, fb, i);
    kahan_add(raw, rawc, raw_p);
    kahan_add(den, denc, den_p);
    // rho = (2 raw) / sqrt(2 den)
    if (act) rho[(size_t)t * p.N_f + k] = den > 0.f ? 1.41421356237309505f * raw * rsqrtf(den) : 0.f;
}

// The method's pair loop: one thread per (template, output bin) over the locked SFTs in
// time order (the separable kernel's records and pipelined loads).  A ring of R_s + 1
// blocks holds, per slot (block mod (R_s + 1), detector), the thread's y and Xi^2
// (thread-private columns of shared memory) and the SFT's prescaled filter weights
// (shared).  A slot that is not a partner of the current SFT -- a block outside the
// window, a gap, a later detector of the current block -- has zero weights, so the
// partner loop is one fixed-length sum without branches.  The filter weights
// Gamma_KL = a^'_K a^'_L + b^'_K b^'_L of the next SFT against every slot are formed once
// per CTA (slot j by thread j mod blockDim) while the ring is updated, so the loop reads
// one shared value per slot.  Before the first SFT of a block the slots of that block
// (and of any skipped block) are cleared.
__global__ void __launch_bounds__(256) demod_pair_kernel(DevParams p, int m_lo, int nbins, int n_blk, int Rs,
                                                         const float2* __restrict__ z,
                                                         const DemodTiming* __restrict__ recs, int n_list,
                                                         const double* __restrict__ dfreq,
                                                         const int64_t* __restrict__ kbar, int64_t t_base,
                                                         float* __restrict__ rho) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int Q = p.Q, W = (Rs + 1) * Q;
    float2* ry = (float2*)sm;                          // [W][nthr] y
    float* rx = (float*)(ry + (size_t)W * nthr);       // [W][nthr] Xi^2
    float2* rab = (float2*)(rx + (size_t)W * nthr);    // [W] (a^', b^'), zero: not a partner
    float* sg = (float*)(rab + W);                     // [W] Gamma of the current SFT per slot
    const int64_t t = t_base + blockIdx.y;
    const int k = blockIdx.x * nthr + tid;
    const bool act = k < (int)p.N_f;
    const DemodTiming* rt = recs + (size_t)(t - t_base) * (n_list + 2);
    for (int j = 0; j < W; ++j) {
        ry[(size_t)j * nthr + tid] = make_float2(0.f, 0.f);
        rx[(size_t)j * nthr + tid] = 0.f;
    }
    for (int j = tid; j < W; j += nthr) {
        rab[j] = make_float2(0.f, 0.f);
        sg[j] = 0.f;                                   // the first SFT has no partner
    }
    if (n_list == 0) {
        if (act) rho[(size_t)t * p.N_f + k] = 0.f;
        return;
    }
    __syncthreads();
    const float df = (float)__ldg(dfreq + (act ? k : 0));
    const int64_t kb = __ldg(kbar + (act ? k : 0));
    const float kh = (float)(kb >> 7), kl = (float)(kb & 127);
    float raw = 0.f, rawc = 0.f, den = 0.f, denc = 0.f;
    auto step = [&](SepRec& Rc, SftIn& Fc, const SepRec& Rn, SftIn& Fn, int i) {
        rec_fetch(Fn, Rn, df, kh, kl, m_lo, nbins, n_blk, z);
        const float a = Rc.t1.y, b = Rc.t1.z;
        const int key = __float_as_int(Rc.t1.w);
        const int l = key >> 2, X = key & 3;
        const int ln = __float_as_int(Rn.t1.w) >> 2;    // block of SFT i + 1 (padding: the last block)
        Rc = load_rec(rt + i + 2);
        float xi2;
        const float2 y = sft_y(Fc, xi2);
        float pr = 0.f, pq = 0.f;
        for (int j = 0; j < W; ++j) {
            const float g = sg[j];
            const float2 yl = ry[(size_t)j * nthr + tid];
            pr = fmaf(g, fmaf(y.x, yl.x, y.y * yl.y), pr);
            pq = fmaf(g * g, rx[(size_t)j * nthr + tid], pq);
        }
        kahan_add(raw, rawc, pr);
        kahan_add(den, denc, xi2 * pq);
        __syncthreads();                               // every thread is done with the ring
        const int bl = l % (Rs + 1), slot = bl * Q + X;
        ry[(size_t)slot * nthr + tid] = y;
        rx[(size_t)slot * nthr + tid] = xi2;
        // the ring's weights after SFT i (its own slot set; SFT i + 1 opening block ln
        // clears the slots of blocks l + 1 .. ln, all of them after R_s + 1 blocks) and
        // Gamma of SFT i + 1 against each slot
        const float an = Rn.t1.y, bn = Rn.t1.z;
        const int jump = ln - l;
        for (int j = tid; j < W; j += nthr) {
            float2 ab = j == slot ? make_float2(a, b) : rab[j];
            if (jump > 0) {
                const int d = j / Q - bl;                 // block-slot distance after l, 0 .. R_s
                const int dd = d <= 0 ? d + Rs + 1 : d;   // 1 .. R_s + 1
                if (dd <= jump) ab = make_float2(0.f, 0.f);
            }
            rab[j] = ab;
            sg[j] = fmaf(an, ab.x, bn * ab.y);
        }
        __syncthreads();
    };
    SepRec ra = load_rec(rt);
    SepRec rb = load_rec(rt + 1);
    SftIn fa, fb;
    rec_fetch(fa, ra, df, kh, kl, m_lo, nbins, n_blk, z);
    int i = 0;
    for (; i + 1 < n_list; i += 2) {
        step(ra, fa, rb, fb, i);
        step(rb, fb, ra, fa, i + 1);
    }
    if (i < n_list) step(ra, fa, rb, fb, i);
    // rho = (2 raw) / sqrt(2 den)
    if (act) rho[(size_t)t * p.N_f + k] = den > 0.f ? 1.41421356237309505f * raw * rsqrtf(den) : 0.f;
}

}  // namespace
}  // namespace cc

using namespace cc;

extern "C" cc_status crosscorr_demod_prepare(cc_plan* plan, const void* const* x_dev, int32_t n_bin,
                                             double doppler_max, void* stream) {
    CC_NVTX_RANGE("crosscorr_demod_prepare");
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (n_bin != 2) return fail(CC_ERR_UNSUPPORTED, "demodulation search implemented for n_bin = 2");
    if (!(doppler_max >= 0) || doppler_max > 0.01) return fail(CC_ERR_INVALID, "doppler_max must be in [0, 0.01]");
    if (doppler_max == 0) doppler_max = 5e-4;
    int64_t nsft = 0;
    {
        const double r = plan->cfg.T_sft / plan->cfg.dt;
        nsft = (int64_t)llround(r);
    }
    if (nsft < 2 || nsft > DM_MAX_SFT_SAMPLES) return fail(CC_ERR_UNSUPPORTED, "T_sft / dt must be 2..16384");
    cc_status s = set_inputs(plan, x_dev);
    if (s != CC_OK) return s;
    const DevParams& p = plan->dp;
    const int64_t n_blk = p.N_t / nsft;
    if (n_blk < 1) return fail(CC_ERR_INVALID, "series shorter than one SFT");
    // bins a signal of the band can reach: |f - f_h| <= max |df| plus Doppler and the kernel
    double dmin = 1e300, dmax = -1e300;
    for (double f : plan->freq) {
        dmin = std::min(dmin, f - plan->cfg.f_h);
        dmax = std::max(dmax, f - plan->cfg.f_h);
    }
    const double Tsft = nsft * plan->cfg.dt;
    const double wing = doppler_max * (plan->cfg.f_h + std::max(std::fabs(dmin), std::fabs(dmax))) * Tsft;
    const int m_lo = (int)std::floor(dmin * Tsft - wing) - 2;
    const int m_hi = (int)std::ceil(dmax * Tsft + wing) + 2;
    const int nbins = m_hi - m_lo + 1;
    if (nbins > nsft) return fail(CC_ERR_UNSUPPORTED, "band plus Doppler wider than an SFT");
    // device arrays (plan-owned; replaced on a new prepare)
    cudaError_t e;
    for (void* ptr : {plan->demod_z, plan->demod_w, plan->demod_tw})
        if (ptr) cudaFree(ptr);
    plan->demod_z = plan->demod_w = plan->demod_tw = nullptr;
    plan->demod_ready = false;
    std::vector<float2> tw(nsft);
    for (int64_t j = 0; j < nsft; ++j) {
        const double a = -2.0 * M_PI * (double)j / (double)nsft;
        tw[j] = make_float2((float)cos(a), (float)sin(a));
    }
    if ((e = cudaMalloc(&plan->demod_tw, sizeof(float2) * nsft)) != cudaSuccess ||
        (e = cudaMalloc(&plan->demod_z, sizeof(float2) * (size_t)p.Q * n_blk * nbins)) != cudaSuccess ||
        (e = cudaMalloc(&plan->demod_w, sizeof(float4) * (size_t)p.Q * n_blk)) != cudaSuccess)
        return cuda_fail(e, "demodulation SFT allocation");
    cudaStream_t st = (cudaStream_t)stream;
    if ((e = cudaMemcpyAsync(plan->demod_tw, tw.data(), sizeof(float2) * nsft, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return cuda_fail(e, "demodulation twiddles");
    const size_t smem = sizeof(float2) * nsft;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(sft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return cuda_fail(e, "sft smem attribute");
    sft_kernel<<<dim3((unsigned)n_blk, (unsigned)p.Q), SFT_THREADS, smem, st>>>(
        p, (int)nsft, m_lo, nbins, (int)n_blk, (const float2*)plan->demod_tw, (float2*)plan->demod_z,
        (float4*)plan->demod_w);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sft_kernel launch");
    // host copies the search needs: output bins' df (FP64) and kbar
    if (!plan->demod_df) {
        if ((e = cudaMalloc(&plan->demod_df, sizeof(double) * plan->N_f)) != cudaSuccess ||
            (e = cudaMalloc(&plan->demod_kbar, sizeof(int64_t) * plan->N_f)) != cudaSuccess)
            return cuda_fail(e, "demodulation bin tables");
        std::vector<double> df(plan->N_f);
        for (int64_t i = 0; i < plan->N_f; ++i)
            df[i] = (plan->f_r - 0.5 / plan->cfg.dt) + (double)plan->kbar[i] / plan->T_FFT;
        if ((e = cudaMemcpy(plan->demod_df, df.data(), sizeof(double) * plan->N_f, cudaMemcpyHostToDevice)) !=
                cudaSuccess ||
            (e = cudaMemcpy(plan->demod_kbar, plan->kbar.data(), sizeof(int64_t) * plan->N_f,
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return cuda_fail(e, "demodulation bin tables");
    }
    // the locked SFTs in time order (key 4 l + X) and each block's first entry, for the
    // separable form
    {
        std::vector<float4> w((size_t)p.Q * n_blk);
        if ((e = cudaMemcpyAsync(w.data(), plan->demod_w, sizeof(float4) * w.size(), cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(e, "demodulation SFT weights");
        std::vector<int> list, boff(n_blk + 1);
        for (int64_t l = 0; l < n_blk; ++l) {
            boff[l] = (int)list.size();
            for (int X = 0; X < p.Q; ++X)
                if (w[(size_t)X * n_blk + l].z != 0.f) list.push_back((int)(4 * l + X));
        }
        boff[n_blk] = (int)list.size();
        for (void* ptr : {plan->demod_list, plan->demod_boff})
            if (ptr) cudaFree(ptr);
        plan->demod_list = plan->demod_boff = nullptr;
        if ((e = cudaMalloc(&plan->demod_list, sizeof(int) * std::max<size_t>(1, list.size()))) != cudaSuccess ||
            (e = cudaMalloc(&plan->demod_boff, sizeof(int) * boff.size())) != cudaSuccess ||
            (!list.empty() && (e = cudaMemcpy(plan->demod_list, list.data(), sizeof(int) * list.size(),
                                              cudaMemcpyHostToDevice)) != cudaSuccess) ||
            (e = cudaMemcpy(plan->demod_boff, boff.data(), sizeof(int) * boff.size(), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
            return cuda_fail(e, "demodulation SFT list");
        plan->demod_nlist = (int)list.size();
    }
    plan->demod_nsft = (int)nsft;
    plan->demod_m_lo = m_lo;
    plan->demod_nbins = nbins;
    plan->demod_nblk = (int)n_blk;
    plan->demod_ready = true;
    return CC_OK;
}

extern "C" cc_status crosscorr_plan_set_demod_form(cc_plan* plan, int form) {
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (form != CC_DEMOD_PAIRS && form != CC_DEMOD_SEPARABLE) return fail(CC_ERR_INVALID, "unknown demodulation form");
    plan->demod_form = form;
    return CC_OK;
}

extern "C" cc_status crosscorr_demod_search(cc_plan* plan, const cc_template* t_dev, int64_t n_t, float* rho_dev,
                                            void* stream) {
    CC_NVTX_RANGE("crosscorr_demod_search");
    if (!plan) return fail(CC_ERR_INVALID, "plan is null");
    if (n_t < 0) return fail(CC_ERR_INVALID, "n_t must be >= 0");
    if (!plan->demod_ready) return fail(CC_ERR_INVALID, "call crosscorr_demod_prepare first");
    if (n_t == 0) return CC_OK;
    if (!t_dev || !rho_dev) return fail(CC_ERR_INVALID, "null device pointer");
    const DevParams& p = plan->dp;
    const int n_blk = plan->demod_nblk, nsft = plan->demod_nsft;
    const double Tsft = nsft * plan->cfg.dt;
    const int Rs = (int)std::floor(plan->cfg.T_max / Tsft + 1e-9);
    const int W = (Rs + 1) * p.Q;
    const bool sep = plan->demod_form == CC_DEMOD_SEPARABLE;
    const int n_list = plan->demod_nlist;
    // separable form: 128 threads, the ring of block sums while it stays within DM_SEP_RING
    const bool sep_ring = sep && (size_t)(Rs + 1) * 7 * 128 * sizeof(float) <= DM_SEP_RING;
    int nthr = sep ? 128 : 256;
    auto ring_bytes = [&](int nt) {
        return sep ? (sep_ring ? (size_t)(Rs + 1) * 7 * nt * sizeof(float) : 0)
                   : (size_t)W * nt * 12 + (size_t)W * 12;
    };
    while (nthr > 32 && ring_bytes(nthr) > DM_RING_BUDGET) nthr /= 2;
    if (ring_bytes(nthr) > DM_RING_BUDGET) return fail(CC_ERR_UNSUPPORTED, "T_max / T_sft too large for the pair ring");
    // exact window sum (over the ring, or recomputed from the bins) after 4 (R_s + 1)
    // single-block steps: the FP32 rounding of the running sums cannot drift further
    const int refresh = 4 * (Rs + 1);
    // timing records for a batch of templates: the list of locked SFTs plus two padding
    const size_t per_t = sizeof(DemodTiming) * ((size_t)n_list + 2);
    const int64_t batch = std::max<int64_t>(1, std::min<int64_t>({n_t, (int64_t)((size_t)2 << 30) / (int64_t)per_t, 65535}));
    if (sep) {
        // CTA size of the separable kernel (every thread does the same work, issue-bound):
        // the fewest resident-thread slots over whole waves of the first batch,
        // ceil(CTAs / (resident CTAs x SMs)) x resident threads per SM
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const void* kern = sep_ring ? (const void*)demod_sep_kernel<true> : (const void*)demod_sep_kernel<false>;
        int64_t best = -1;
        for (int nt : {128, 96, 64}) {
            int occ = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, ring_bytes(nt)) != cudaSuccess || occ < 1)
                continue;
            const int64_t ctas = (plan->N_f + nt - 1) / nt * std::min(batch, n_t);
            const int64_t est = (ctas + (int64_t)occ * sms - 1) / ((int64_t)occ * sms) * occ * nt;
            if (best < 0 || est < best) {
                best = est;
                nthr = nt;
            }
        }
    }
    cc_status s = ensure_workspace(plan, per_t * batch);
    if (s != CC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    const size_t smem = ring_bytes(nthr);
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(sep ? (const void*)demod_sep_kernel<true> : (const void*)demod_pair_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return cuda_fail(e, "demodulation smem attribute");
    const double df0 = plan->f_r - 0.5 / plan->cfg.dt, dK = 1.0 / plan->T_FFT;
    for (int64_t t0 = 0; t0 < n_t; t0 += batch) {
        const int64_t nb = std::min(batch, n_t - t0);
        if (n_list > 0) {
            demod_timing_list_kernel<<<dim3((unsigned)((n_list + 2 + 127) / 128), (unsigned)nb), 128, 0, st>>>(
                p, t_dev + t0, nsft, n_blk, df0, dK, (const int*)plan->demod_list, n_list,
                (const float4*)plan->demod_w, (DemodTiming*)plan->ws);
            count_launch();
        }
        cudaEvent_t ev0, ev1;   // diagnostic timing of the pair loop (crosscorr_plan_set_kernel_timing)
        timing_pair(plan, &ev0, &ev1);
        if (ev0) cudaEventRecord(ev0, st);
        const dim3 grid((unsigned)((plan->N_f + nthr - 1) / nthr), (unsigned)nb);
        if (sep)
            (sep_ring ? demod_sep_kernel<true> : demod_sep_kernel<false>)<<<grid, nthr, smem, st>>>(
                p, plan->demod_m_lo, plan->demod_nbins, n_blk, Rs, refresh, (const float2*)plan->demod_z,
                (const DemodTiming*)plan->ws, n_list, (const int*)plan->demod_boff, (const double*)plan->demod_df,
                (const int64_t*)plan->demod_kbar, t0, rho_dev);
        else
            demod_pair_kernel<<<grid, nthr, smem, st>>>(
                p, plan->demod_m_lo, plan->demod_nbins, n_blk, Rs, (const float2*)plan->demod_z,
                (const DemodTiming*)plan->ws, n_list, (const double*)plan->demod_df,
                (const int64_t*)plan->demod_kbar, t0, rho_dev);
        count_launch();
        if (ev1) cudaEventRecord(ev1, st);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? CC_OK : cuda_fail(e, "demodulation launch");
}
