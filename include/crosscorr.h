/*
 * crosscorr.h -- C ABI of the GB300 resampled cross-correlation (CrossCorr) library.
 *
 * The library computes, for a batch of binary-orbit templates (a_p, T_asc, P),
 * the normalised cross-correlation statistic rho(f) of Meadors, Krishnan, Papa,
 * Whelan & Zhang, "Resampling to accelerate cross-correlation searches for
 * continuous gravitational waves from binary systems":
 *
 *   1. resample each detector's heterodyned complex series into the source
 *      frame (Sec. III A: Eqs. t-ssb-equation, tau-equation, the windowed-sinc
 *      formula shannon-interp-formula and resampled-time-series-q-eq) and weight
 *      it by the antenna/noise functions (Eq. norm-a-eq);
 *   2. take zero-padded FFTs segment by segment at the metric resolution and
 *      keep the decimated output bins (Sec. III B 3-4);
 *   3. sum the weighted cross-correlation over all detector/segment pairs with
 *      lag up to T_max and normalise (Sec. III B 1 and Eq. final-formatted-rho).
 *
 * Conventions for every entry point
 *   - Times are seconds.  cc_config.t0 is the GPS time of sample 0 and the
 *     origin of the source-frame grid tau_r = t0 + r*dt; all table times in
 *     cc_detector are relative to t0.  Template T_asc is absolute GPS.
 *   - "host" pointers are read during the call only (the plan copies what it
 *     keeps); "device" pointers are CUDA global memory owned by the caller and
 *     must stay valid until the work queued on the stream has finished.
 *   - Complex values are interleaved float pairs (re, im), 8 bytes each.
 *   - Every call is asynchronous on the given stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream) except crosscorr_plan,
 *     crosscorr_plan_info, crosscorr_plan_destroy and crosscorr_rho_topk
 *     (which waits for its host copy).
 *   - Errors are returned, never raised or aborted on.  CC_ERR_INVALID for bad
 *     arguments (checked before any work is queued), CC_ERR_OOM when device
 *     memory cannot be allocated, CC_ERR_CUDA when a CUDA call fails,
 *     CC_ERR_UNSUPPORTED for valid but unimplemented options.  The message of
 *     the last failure on the calling thread is returned by
 *     crosscorr_last_error().
 *   - A plan is not thread-safe: use one plan per host thread / stream.
 */
#ifndef CROSSCORR_H
#define CROSSCORR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CC_OK = 0,
    CC_ERR_INVALID = 1,
    CC_ERR_OOM = 2,
    CC_ERR_CUDA = 3,
    CC_ERR_TIMEOUT = 4,
    CC_ERR_UNSUPPORTED = 5
} cc_status;

/* Pair sets (Sec. III B 1, pair selection for the resampled statistic). */
enum {
    CC_PAIRS_UNORDERED = 0,   /* each unordered pair once: X<Y with |K-L|<=R, and X=Y with
                                 1<=L-K<=R (auto-correlation excluded) -- the default */
    CC_PAIRS_CROSS_ONLY = 1,  /* X<Y with |K-L|<=R only (radiometer-like option) */
    CC_PAIRS_ALL_ORDERED = 2  /* every ordered pair with |K-L|<=R incl. K=L, X=Y
                                 (the F-statistic limit of Appendix A) */
};

enum { CC_INTERP_EXACT = 0, CC_INTERP_LEARNED = 1 };
enum { CC_STORE_FP32 = 0, CC_STORE_BF16 = 1 };

#define CC_MAX_DET 4

/* Search set-up of one frequency band. */
typedef struct {
    double t0;        /* GPS time of sample 0 and origin of the source-frame grid */
    double dt;        /* sampling interval dt' of the heterodyned series */
    double f_h;       /* heterodyne frequency = band centre [Hz] */
    double f_band;    /* searched band width [Hz] */
    double T_sft;     /* noise-estimation block [s]; integer multiple of dt */
    double T_short;   /* segment length [s]; 0 selects max(T_max, T_sft); integer multiple of dt */
    double T_max;     /* maximum lag [s]; R = floor(T_max / T_short) */
    double mu_f;      /* frequency mismatch for the metric spacing (0.1 typical) */
    int32_t n_det;    /* Q, 1..CC_MAX_DET */
    int32_t D;        /* windowed-sinc half width: 2D+1 taps, 1..32 */
    int32_t interp;   /* CC_INTERP_EXACT, or CC_INTERP_LEARNED (then call
                         crosscorr_plan_set_learned_interp before any compute call) */
    int32_t store;    /* CC_STORE_FP32 or CC_STORE_BF16 for the resampled a_r, b_r series */
    int32_t pair_mode;/* CC_PAIRS_* */
    int32_t reserved;
    int64_t n_samples;/* N_t samples per detector */
} cc_config;

/* Per-detector inputs (host memory; copied by crosscorr_plan). */
typedef struct {
    const double* ssb_delay; /* Roemer delay r(t).n/c = t_SSB - t [s] at eph_t0 + n*eph_dt,
                                linearly interpolated (Eq. t-ssb-equation) */
    double eph_t0, eph_dt;
    int64_t n_eph;           /* >= 2 */
    const double* a_tab;     /* antenna function a(t) at ab_t0 + n*ab_dt, linearly interpolated */
    const double* b_tab;     /* antenna function b(t), same grid */
    double ab_t0, ab_dt;     /* ab_t0 and ab_dt integer multiples of dt */
    int64_t n_ab;            /* >= 2 */
    const double* sigma;     /* noise std per T_sft block starting at t = 0; 0 marks a gap */
    int64_t n_sigma;
} cc_detector;

/* One orbital template (Sec. II A 2, Eqs. solve-for-E, Kepler-equation).  The binary
 * Roemer delay at SSB time u is R/c = a_p [sin w (cos E - e) + cos w sqrt(1 - e^2) sin E]
 * with E - e sin E = 2 pi (u - T_p) / P, the periapsis time T_p placed so that the
 * ascending node (true anomaly -w) falls at T_asc.  e = 0 is the circular orbit
 * R/c = a_p sin(2 pi (u - T_asc) / P) (w then has no effect).  0 <= e < 0.95. */
typedef struct {
    double a_p;    /* projected semi-major axis a sin i / c [s] */
    double T_asc;  /* time of ascension, GPS [s] */
    double P;      /* orbital period [s] */
    double e;      /* eccentricity */
    double omega;  /* argument of periapsis w [rad] */
} cc_template;

/* One top-k record. */
typedef struct {
    int64_t tmpl;  /* template index within the rho array */
    int32_t bin;   /* output bin k, 0..N_f-1 */
    int32_t pad;
    double freq;   /* absolute frequency of the bin [Hz] */
    float rho;
    float pad2;
} cc_hit;

/* Plan quantities (Sec. III B 3-4), returned by crosscorr_plan_info. */
typedef struct {
    int64_t N_s;      /* samples per T_short segment */
    int64_t M;        /* number of segments, floor(N_t / N_s) */
    int64_t R;        /* T_max / T_short */
    int64_t N_tau;    /* M * N_s resampled samples per detector */
    int64_t N_FFT;    /* 2^ceil(log2 N_FFT0) */
    int64_t N_f;      /* output bins, floor(f_band / delta-lambda_f) */
    int64_t k0;       /* FFT bin of f_h - f_band/2 (FFT indexed from f_FFT) */
    int64_t L;        /* coset FFT length used on chip */
    int64_t C;        /* number of cosets, N_FFT / L */
    double T_coh, dlf, N_FFT0, T_FFT, nu_R, f_r, f_FFT;
    size_t ws_bytes;  /* device workspace currently held by the plan */
} cc_plan_info;

typedef struct cc_plan cc_plan;

/* Build a plan: validates cfg, derives T_short, T_coh, delta-lambda_f, N_FFT,
 * nu_R, f_r*, k0 and the output bins k-bar(k) = k0 + floor(nu_R k) (Sec. III B 3-4
 * with the readings listed in the design notes), copies the detector tables
 * to the device.  dets: host array of cfg->n_det detectors.  *out receives a
 * plan owned by the caller and released with crosscorr_plan_destroy. */
cc_status crosscorr_plan(const cc_config* cfg, const cc_detector* dets, cc_plan** out);

/* Learned 8-tap interpolator.  The paper has no counterpart: it is a stand-in for the
 * 2D+1-tap windowed sinc of Eq. shannon-interp-formula.  A network maps the fractional
 * offset u = t/dt' - floor(t/dt') in [0, 1) and the band half-width nu_c (cycles per
 * sample; the local spectral context) to 8 taps c_0..c_7:
 *   s  = (2u - 1, (2 nu_c - nu_lo - nu_hi) / (nu_hi - nu_lo))
 *   h1 = tanh(s W1 + b1),  h2 = tanh(h1 W2 + b2),  c = h2 W3 + b3
 *   x(t) = sum_n c_n x[floor(t/dt') - 3 + n]     (samples outside [0, N_t) are zero)
 * Weights are BF16 bit patterns, concatenated row-major in the order
 *   W1 [2][64], b1 [64], W2 [64][64], b2 [64], W3 [64][8], b3 [8]   (4872 values),
 * W[i][o] multiplying input i into output o.  The network is evaluated with FP32
 * accumulation; the plan tabulates the taps on a fine grid of u (1025 nodes) once and
 * interpolates them linearly in u per sample. */
#define CC_LEARNED_N_WEIGHTS 4872
typedef struct {
    const uint16_t* weights_bf16;  /* host, CC_LEARNED_N_WEIGHTS values; copied */
    int64_t n_weights;             /* must equal CC_LEARNED_N_WEIGHTS */
    double nu_lo, nu_hi;           /* nu_c range the network was trained for (nu_lo < nu_hi) */
    double nu_c;                   /* this plan's band half-width, within [nu_lo, nu_hi] */
} cc_learned_interp;

/* Install the learned interpolator in a plan built with interp = CC_INTERP_LEARNED
 * (CC_ERR_INVALID otherwise, or on a wrong weight count, a non-finite weight or an
 * inverted range; CC_ERR_UNSUPPORTED if nu_c is outside [nu_lo, nu_hi]).  Synchronous:
 * uploads the weights and tabulates the taps on the device before returning.  May be
 * called again to replace the weights. */
cc_status crosscorr_plan_set_learned_interp(cc_plan* plan, const cc_learned_interp* li);

/* Plan quantities; freqs_host (nullable, N_f doubles) receives the absolute
 * output frequencies f_FFT + k-bar/T_FFT, kbar_host (nullable, N_f int64) the bins. */
cc_status crosscorr_plan_info(const cc_plan* plan, cc_plan_info* info, double* freqs_host,
                              int64_t* kbar_host);

/* Stage 1, resample and weight (Eqs. tau-equation, resampled-time-series-q-eq,
 * norm-a-eq): for template t and detector X writes
 *   ab[((t*Q + X)*2 + 0)*N_tau + r] = a_r = alpha_r x'_r exp(-2 pi i f_r* tau_r)
 *   ab[((t*Q + X)*2 + 1)*N_tau + r] = b_r = beta_r  x'_r exp(-2 pi i f_r* tau_r)
 * with x'_r the heterodyne-corrected windowed-sinc interpolation at t(tau_r) and
 * alpha = a/sigma^2, beta = b/sigma^2 at that detector time (0 in gaps), and
 *   norm[((t*Q + X)*M + K)*4 + {0,1,2}] = sum over segment K of
 *   alpha^2 sigma^2, beta^2 sigma^2, alpha beta sigma^2   (hat-A, hat-B, hat-C).
 * x_dev: host array of Q device pointers to complex64[N_t].  t_dev: device
 * cc_template[n_t].  ab_dev: device complex64 (store = FP32) or bf16 pairs
 * (store = BF16) [n_t][Q][2][N_tau].  norm_dev: device float[n_t][Q][M][4].
 * The FP64 timing knots of up to 8 GB of templates at a time are kept in the plan's
 * workspace (grown as needed; a caller-owned workspace too small for one template's
 * knots makes every block compute its own).  Samples of a segment over which a
 * detector's noise blocks are all gaps are written as exact zeros. */
cc_status crosscorr_resample(cc_plan* plan, const void* const* x_dev, const cc_template* t_dev,
                             int64_t n_t, void* ab_dev, float* norm_dev, void* stream);

/* Stage 2, segment spectra (Eqs. fft-inklings to the F-bar definitions): for each
 * template, detector X, segment K and weight w in {a, b}
 *   F[(((t*Q + X)*M + K)*2 + w)*N_f + k] = sum_{r in segment K} w_r exp(-2 pi i (k-bar_k - N_FFT/2) r / N_FFT)
 * i.e. the zero-padded N_FFT-point transform at the selected bins with the
 * segment-start phase Phi_in included.  ab_dev as written by stage 1; F_dev:
 * device complex64[n_t][Q][M][2][N_f].  Asynchronous on `stream`; on 4096-point cosets
 * (Q <= 2, whole segments) it uses a plan-owned unit counter, so two calls on one plan
 * must not run concurrently on different streams (as for every call on a plan). */
cc_status crosscorr_segment_fft(cc_plan* plan, const void* ab_dev, int64_t n_t, void* F_dev,
                                void* stream);

/* Stage 3, pair sum and normalisation (Sec. III B 1, Eq. final-formatted-rho):
 *   rho[t*N_f + k] = sqrt(2) Re sum_P [conj(F_a,XK) F_a,YL + conj(F_b,XK) F_b,YL]
 *                    / sqrt(sum_P (A_XK A_YL + B_XK B_YL + 2 C_XK C_YL))
 * over the pair set of cfg.pair_mode, accumulated in compensated FP32.
 * F_dev, norm_dev as written by stages 1-2; rho_dev: device float[n_t][N_f]. */
cc_status crosscorr_pair_accumulate(cc_plan* plan, const void* F_dev, const float* norm_dev,
                                    int64_t n_t, float* rho_dev, void* stream);

/* Whole path fused on chip: the same rho as stages 1-3 without materialising
 * a_r, b_r or F.  Inputs and output as for stages 1 and 3. */
cc_status crosscorr_search(cc_plan* plan, const void* const* x_dev, const cc_template* t_dev,
                           int64_t n_t, float* rho_dev, void* stream);

/* crosscorr_search for callers that cannot allocate device memory while searching:
 * for example a service that hands all device memory to its own pool at start-up and
 * forbids later cudaMalloc/cudaFree (which may also synchronise the device and stall
 * its other streams).  The paper has no counterpart; this is an engineering variant.
 * Same inputs, output and result as crosscorr_search; it never allocates.  Its only
 * scratch (one double per template) is a fixed 512 KiB array compiled into the library,
 * which every GPU that loads the library holds until the process exits:
 *   - n_t may be at most 65536 (CC_ERR_INVALID above that; split the batch);
 *   - plans that need the staged path (BF16 storage, very long segments) return
 *     CC_ERR_UNSUPPORTED;
 *   - the first call on a device looks up the array's device address with that device
 *     current, so make that first call before any stream capture; after a device reset
 *     (cudaDeviceReset or another teardown of the primary context) the array is reloaded,
 *     possibly at another address, and the next call looks it up again, so that call too
 *     must come before any capture;
 *   - every call shares the array and it keeps the last call's contents; each call
 *     overwrites the entries it uses before reading them, so nothing needs clearing,
 *     but calls that overlap on the GPU (other streams, other host threads) race on it
 *     and must be serialised by the caller. */
cc_status crosscorr_search_noalloc(cc_plan* plan, const void* const* x_dev, const cc_template* t_dev,
                                   int64_t n_t, float* rho_dev, void* stream);

/* How crosscorr_search computes rho (all give the same rho to rounding):
 *   CC_PATH_AUTO      the fastest path the plan supports (the default): TWO_PASS, else
 *                     FUSED, else STAGED;
 *   CC_PATH_FUSED     one kernel per template batch: a thread-block cluster resamples
 *                     each segment into shared memory and transforms it on chip; needs
 *                     a few MB of workspace (FP32 storage, coset length <= 4096);
 *   CC_PATH_TWO_PASS  a_r, b_r of a template batch written to HBM in the plan's
 *                     storage type (up to 24 GB of workspace), then one CTA per
 *                     (coset, weight) transforms each segment and folds it into the
 *                     pair sum on chip (Q <= 2, R <= 1, not CC_PAIRS_CROSS_ONLY, coset
 *                     length >= 64, output bins in the lower half of each coset); for
 *                     coset length 4096 with whole segments this is a persistent kernel
 *                     fed by TMA bulk copies (see crosscorr_plan_check);
 *   CC_PATH_STAGED    the three stage kernels with spectra in HBM (any plan). */
enum { CC_PATH_AUTO = 0, CC_PATH_FUSED = 1, CC_PATH_TWO_PASS = 2, CC_PATH_STAGED = 3 };

/* Select the path of crosscorr_search (CC_ERR_INVALID for an unknown value,
 * CC_ERR_UNSUPPORTED if the plan does not fit it). */
cc_status crosscorr_plan_set_path(cc_plan* plan, int path);

/* The path crosscorr_search takes for this plan (never CC_PATH_AUTO). */
cc_status crosscorr_plan_search_path(const cc_plan* plan, int* path);

/* Device workspace.  crosscorr_search keeps its scratch (knot records, partial sums, and
 * on the two-pass and staged paths the resampled series) in a workspace that the plan
 * allocates and grows on demand.  crosscorr_plan_set_workspace hands it caller-owned
 * device memory instead (ws_dev 256-byte aligned, kept until replaced; NULL returns to
 * plan-owned memory): a search that needs more than ws_bytes fails with CC_ERR_OOM and
 * allocates nothing, which makes crosscorr_search capturable in a CUDA graph.  Plans
 * whose searches run one after another on one stream may share one workspace.
 * crosscorr_plan_workspace_size gives the bytes a search of n_t templates needs on the
 * path crosscorr_search takes, with the plan's current tuning. */
cc_status crosscorr_plan_set_workspace(cc_plan* plan, void* ws_dev, size_t ws_bytes);
cc_status crosscorr_plan_workspace_size(const cc_plan* plan, int64_t n_t, size_t* bytes);

/* Work-split tuning of crosscorr_search (results do not depend on it). */
typedef struct {
    int64_t batch_templates;  /* two-pass: templates per resample/spectrum batch
                                 (0: as many as 24 GB of resampled series hold) */
    int32_t chunk_waves;      /* fused and two-pass: split each template's segments into
                                 chunks until the launch has about this many CTA waves
                                 (0: 4 for fused, 40 for two-pass) */
    int32_t transform_len;    /* two-pass, segments of at most 4096 samples: 0 takes the
                                 plan's coset length (the power of two covering a segment),
                                 4096 the persistent kernel's 4096-point coset transforms
                                 with the segment zero-padded (needs N_FFT >= 4096: fewer
                                 cosets, more transform work, a faster kernel) */
} cc_tuning;
cc_status crosscorr_plan_set_tuning(cc_plan* plan, const cc_tuning* tuning);

/* Detector-frame ("demodulation") CrossCorr, the statistic the resampled method replaces
 * (Sec. II: Eqs. fourier-transform-def, normalized-z-bin, total-data-eq, geometric-filter,
 * norm-cc, textbook-cc-rho), at the plan's output frequencies on the same data, for
 * comparison.  SFTs are the locked T_sft blocks (T_sft / dt in 2..16384 samples);
 * Gamma^ave_KL pairs every two distinct SFTs whose mid-times differ by at most T_max
 * (each unordered pair once); n_bin = 2 sinc-weighted bins per SFT; each pair is
 * weighted by Xi_K Xi_L and N normalises rho to unit variance in noise.
 *
 * crosscorr_demod_prepare computes the SFT bins a signal of the band can reach for
 * Doppler factors |dtau/dt - 1| <= doppler_max (0 selects 5e-4) from x_dev (Q device
 * pointers to complex64[N_t], as for crosscorr_search) into plan-owned device memory, and
 * the time-ordered list of locked SFTs the search walks; it synchronises `stream` once
 * (the lock flags come back to the host to build that list).  crosscorr_demod_search
 * then writes rho to rho_dev[n_t][N_f] (device) for device templates t_dev[n_t],
 * asynchronously on `stream`, with per-template SFT records (32 bytes per locked SFT) in
 * the plan workspace, grown on demand. */
cc_status crosscorr_demod_prepare(cc_plan* plan, const void* const* x_dev, int32_t n_bin, double doppler_max,
                                  void* stream);
cc_status crosscorr_demod_search(cc_plan* plan, const cc_template* t_dev, int64_t n_t, float* rho_dev,
                                 void* stream);

/* How crosscorr_demod_search sums the pairs (the same rho up to FP32 rounding):
 *   CC_DEMOD_PAIRS      the method's pair loop, one term per partner SFT (the default; its
 *                       cost per pair is what the paper's comparison with resampling rests on);
 *   CC_DEMOD_SEPARABLE  the geometric filter Gamma_KL = (a^_K a^_L + b^_K b^_L)/10 factored
 *                       into running window sums of a^_L y_L, b^_L y_L and Xi_L^2-weighted
 *                       a^_L^2, a^_L b^_L, b^_L^2: O(1) per SFT.  An algebraic rearrangement
 *                       of Eqs. geometric-filter and textbook-cc-rho, not a form the paper uses. */
enum { CC_DEMOD_PAIRS = 0, CC_DEMOD_SEPARABLE = 1 };
cc_status crosscorr_plan_set_demod_form(cc_plan* plan, int form);

/* Input preparation (Appendix B): the heterodyned, downsampled series the search starts
 * from, built from short Fourier transforms.  band_dev: device complex64 [n_sft][n_prime],
 * the SFT bins k_h - n_prime/2 .. k_h + n_prime/2 - 1 of each SFT (DFT times dt, Eq.
 * fourier-transform-def) around the heterodyne bin k_h = f_h T_sft (f_h on a bin);
 * block_sft_dev: device int64 [n_blocks], the SFT of T_sft block b (block b starts at
 * b T_sft after the series origin), -1 for a gap.  x_dev: device complex64
 * [n_blocks * n_prime] at dt' = T_sft / n_prime:
 *   x(b T_sft + j dt') = exp(-2 pi i f_h b T_sft) (-1)^j
 *                        sum_{m < n_prime} exp(2 pi i j m / n_prime) band[b][m] / T_sft
 * (Eqs. shifted-for-fft, long-time-series-het-corrected), zero in gaps.  Asynchronous on
 * `stream` (a small twiddle table is allocated stream-ordered).  1 <= n_prime <= 16384. */
cc_status crosscorr_sfts_to_series(const void* band_dev, const int64_t* block_sft_dev, int64_t n_blocks,
                                   int64_t n_prime, double T_sft, double f_h, void* x_dev, void* stream);

/* Template placement (Sec. III A; host functions, no GPU).  crosscorr_metric: the
 * phase-mismatch metric g [3][3] (row-major, for lambda = (a_p, T_asc, P)) of Eq.
 * phase-derivs-metric, g_ij = 1/2 < d(Phi_K - Phi_L)/d lambda^i d(Phi_K - Phi_L)/d lambda^j >
 * over the pairs of the detector-frame statistic: SFT mid-times (k + 1/2) T_sft,
 * k < floor(T_obs / T_sft), every unordered pair of distinct SFTs of the Q detectors within
 * T_max (same-time pairs of two detectors have zero phase difference), for the circular
 * orbit `orbit` (host; e must be 0) at frequency f; times relative to t0.
 * crosscorr_lattice: the cubic lattice of Eq. metric-spacing-eq, spacing sqrt(mu / g_ii)
 * from lo[i] covering [lo[i], hi[i]], written to out (host, capacity entries; circular
 * templates, P varying fastest: out[(ia * nT + iT) * nP + iP]); *n_out receives the
 * lattice size (out = NULL queries it). */
cc_status crosscorr_metric(double T_obs, double T_sft, double T_max, int32_t Q, double f, const cc_template* orbit,
                           double t0, double* g);
cc_status crosscorr_lattice(const double* g, double mu, const double* lo, const double* hi, cc_template* out,
                            int64_t capacity, int64_t* n_out);

/* Device-side status of the plan's kernels.  Kernels that wait on asynchronous copies
 * (the persistent spectrum kernel of the two-pass path waits on its TMA bulk copies)
 * bound every wait to about one second; a wait that runs out sets a device error word of
 * the plan and the kernel returns early.  This call synchronises `stream`, reads the
 * word, clears it and returns CC_ERR_TIMEOUT if it was set (the rho of every search since
 * the previous check is then invalid), else CC_OK.  crosscorr_rho_topk makes the same
 * check.  No counterpart in the paper: error reporting of this implementation. */
cc_status crosscorr_plan_check(cc_plan* plan, void* stream);

/* Diagnostic for the bounded waits (no counterpart in the paper): with on != 0, every CTA
 * of the persistent spectrum kernel leaves the bulk copy of its first transform unissued,
 * so that wait runs out after about one second; the CTA records the timeout and returns
 * (no fault, no hang) and crosscorr_plan_check then reports CC_ERR_TIMEOUT.  The rho of
 * such a search is invalid.  Off (0) by default; for tests of the error path. */
cc_status crosscorr_plan_set_wait_test(cc_plan* plan, int on);

/* The k largest rho over (template, bin) of a device float[n_t][N_f] array,
 * descending, ties by (template, bin) ascending; hits_host receives
 * min(k, n_t*N_f) records.  Synchronises the stream.  1 <= k <= 4096.
 * Its candidate lists live in a plan-owned buffer of about 15 MB, allocated by the
 * first call on the plan (later calls allocate nothing) and separate from the search
 * workspace, so a search queued on another stream for the same plan is not disturbed;
 * two top-k calls on one plan must not run at the same time (one plan per thread). */
cc_status crosscorr_rho_topk(cc_plan* plan, const float* rho_dev, int64_t n_t, int k,
                             cc_hit* hits_host, void* stream);

/* Release the plan and everything it owns (NULL is ignored). */
void crosscorr_plan_destroy(cc_plan* plan);

const char* crosscorr_status_string(cc_status s);

/* Message of the last failed call on this thread ("" if none). */
const char* crosscorr_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far (a
 * diagnostic counter, incremented on the host at every launch). */
uint64_t crosscorr_kernel_launches(void);

/* Diagnostic timing of the search's dominant kernel (off by default).  While on, each
 * launch of the spectrum + pair-sum kernel (two-pass path), of the one-pass kernel
 * (fused path, crosscorr_search_noalloc) or of the pair-loop kernel of
 * crosscorr_demod_search is bracketed by a pair of CUDA events recorded on the launching
 * stream (the knot pre-pass, the resampling kernel and the final
 * normalisation pass are outside the pair).  Turning it off keeps the pending records. */
cc_status crosscorr_plan_set_kernel_timing(cc_plan* plan, int on);

/* Total device time of the timed launches recorded since the last call, in ms, and
 * their number; waits for those launches to finish, then clears the record. */
cc_status crosscorr_plan_kernel_time(cc_plan* plan, double* ms, int64_t* launches);

/* Diagnostic: the measured FP32 fused-multiply-add throughput of the current device in
 * TFLOP/s (2 flop per FMA), from a full-occupancy grid of independent FMA chains timed
 * with CUDA events on `stream` (best of three launches after one warm-up; synchronises
 * the stream, about 0.1 s).  The spectrum kernels are bound by the plain FP32 pipes and
 * report their fraction of this figure.  No counterpart in the paper. */
cc_status crosscorr_measure_fp32_peak(double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CROSSCORR_H */
