"""Plain FP64 NumPy restatement of the resampled cross-correlation statistic.

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py.  Slow on purpose; nothing here is blocked, fused or
reordered beyond what the paper's definitions state.

Notation follows the paper (Meadors, Krishnan, Papa, Whelan, Zhang,
"Resampling to accelerate cross-correlation searches for continuous
gravitational waves from binary systems"):

* tau_r = t0 + r dt' is the uniform source-frame grid shared by all detectors
  (Sec. III B 2: resampled series indexed by r; a common epoch makes the
  detector-epoch shift Phi_out vanish).
* tau(t) = t_SSB - a_p sin(Omega (t_SSB - T_asc)), t_SSB = t + r.n/c
  (Eqs. t-ssb and tau with the circular-orbit Roemer delay, Sec. II A 2).
* x'_r = exp(-2 pi i f_h [tau_r - t(tau_r)]) x'(t(tau_r)) with x' interpolated
  by the windowed-sinc (Shannon) formula with 2D+1 Hamming-windowed taps
  (Eqs. shannon-interp-formula, resampled-time-series-q-eq).
* a_r, b_r = (a, b)(t_r) x'_r / sigma^2(t_r) at the detector time t_r = t(tau_r)
  of each source sample (Eq. norm-a-eq; constant factors that cancel in the
  normalised statistic are dropped).
* Per-segment spectra F_a,XK, F_b,XK at the published frequencies (Eqs.
  fft-inklings to the definition of F-bar, with Phi_in included through the
  common-epoch phase).
* rho_k = sqrt(2) Re sum_pairs [conj(F_aK) F_aL + conj(F_bK) F_bL] /
  sqrt(A^2 + 2C^2 + B^2) (Eq. final-formatted-rho with the hat-A/B/C sums of
  Appendix A).

Readings of passages that are silent, garbled or ambiguous are numbered as in
the design notes (reading 1 ... 9) where they are used.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

PAIR_UNORDERED = 0     # reading 6: every unordered pair once, auto-correlation excluded
PAIR_CROSS_ONLY = 1    # radiometer-like option: cross-detector pairs only (Sec. III B 3)
PAIR_ALL_ORDERED = 2   # every ordered pair incl. auto-correlation (F-statistic limit, App. A)

N_FIXED_POINT = 8      # iterations of each timing fixed point (contraction ~1e-4 per step)


# ---------------------------------------------------------------------------
# S0: plan  (Sec. III B 2-4: T_coh, delta-lambda_f, N_FFT, nu_R, f_r*, k0)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Plan:
    dt: float
    N_t: int
    T_short: float
    N_s: int          # samples per T_short segment
    R: int            # T_max / T_short
    M: int            # number of segments
    T_coh: float
    dlf: float        # delta-lambda_f
    N_FFT0: float
    N_FFT: int
    T_FFT: float
    nu_R: float
    N_f: int
    f_r: float        # f_r*
    f_FFT: float
    k0: int
    kbar: np.ndarray  # int64 [N_f]
    freq: np.ndarray  # float64 [N_f], absolute frequency of each output bin
    dfreq: np.ndarray  # float64 [N_f], freq - f_h evaluated without cancellation


def paper_remainder(a: float, b: float) -> float:
    """remainder(a, b) = a - sgn(a) floor(|a|/|b|) |b| (reading 7: the printed
    definition drops the final |b|, without which the result is not a remainder)."""
    if a == 0.0:
        return 0.0
    return a - math.copysign(1.0, a) * math.floor(abs(a) / abs(b)) * abs(b)


def make_plan(cfg, n_fft: Optional[int] = None) -> Plan:
    """Frequency resolution, FFT size and output-bin selection.

    * T_short = max(T_max, T_sft) unless given; R = T_max / T_short
      (Sec. III B 1, pair selection; performance is best with T_short = T_max).
    * T_coh = 2 T_max + T_short (Eq. lag-time constraint and T_coh definition).
    * delta-lambda_f = sqrt(6 mu_f / pi) / T_coh (metric spacing, Sec. III B 3).
    * N_FFT0 = (Delta f_load / delta-lambda_f) ceil(delta-lambda_f T_coh),
      N_FFT = 2^ceil(log2 N_FFT0) (Eq. n-fft-final), with Delta f_load = 1/dt'
      the band the complex series represents.
    * nu_R = delta-lambda_f dt' N_FFT; k-bar(k) = k0 + floor(nu_R k)
      (reading 9: "lround ... to the integer less than its argument" is floor).
    * f_r* = remainder(-f_band/2, 1/T_FFT) (reading 7);
      f_FFT = f_h + f_r* - Delta f_s/2 with Delta f_s = 1/dt' (reading 8: the
      printed f_band T_FFT is not a frequency); k0 places f_h - f_band/2 on
      bin k0.  N_f = floor(f_band / delta-lambda_f) output frequencies.

    ``n_fft`` overrides the power-of-two rule (used only by tests of the
    recovered-power averages, which the paper quotes for T_FFT = 1, 2, 3 T_coh).
    """
    dt = float(cfg.dt)
    T_short = float(cfg.T_short) if cfg.T_short > 0 else max(float(cfg.T_max), float(cfg.T_sft))
    N_s = int(round(T_short / dt))
    if abs(N_s * dt - T_short) > 1e-9 * T_short or N_s < 1:
        raise ValueError("T_short must be a positive integer multiple of dt")
    R = int(math.floor(cfg.T_max / T_short + 1e-9))
    M = int(cfg.n_samples) // N_s
    T_coh = 2.0 * cfg.T_max + T_short
    dlf = math.sqrt(6.0 * cfg.mu_f / math.pi) / T_coh
    df_load = 1.0 / dt
    N_FFT0 = (df_load / dlf) * math.ceil(dlf * T_coh)
    if n_fft is None:
        N_FFT = 1
        while N_FFT < N_FFT0:
            N_FFT *= 2
    else:
        N_FFT = int(n_fft)
    T_FFT = N_FFT * dt
    nu_R = dlf * dt * N_FFT
    N_f = int(math.floor(cfg.f_band / dlf))
    f_r = paper_remainder(-cfg.f_band / 2.0, 1.0 / T_FFT)
    f_FFT = cfg.f_h + f_r - 0.5 / dt
    # k0 = floor((f_h - f_band/2 - f_FFT) T_FFT); the argument is an integer in exact
    # arithmetic, so a 1e-9 guard keeps rounding from moving it one bin down.
    k0 = int(math.floor((cfg.f_h - cfg.f_band / 2.0 - f_FFT) * T_FFT + 1e-9))
    k = np.arange(N_f, dtype=np.float64)
    kbar = k0 + np.floor(nu_R * k).astype(np.int64)
    freq = f_FFT + kbar / T_FFT
    dfreq = (f_r - 0.5 / dt) + kbar / T_FFT
    return Plan(dt, int(cfg.n_samples), T_short, N_s, R, M, T_coh, dlf, N_FFT0, N_FFT,
                T_FFT, nu_R, N_f, f_r, f_FFT, k0, kbar, freq, dfreq)


# ---------------------------------------------------------------------------
# S1: timing  (Eqs. t-ssb-equation, tau-equation, circular Roemer delay)
# ---------------------------------------------------------------------------
def _lerp(t0: float, dt: float, tab: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Linear interpolation of a uniformly sampled table (end intervals extrapolate)."""
    u = (np.asarray(t, np.float64) - t0) / dt
    i = np.clip(np.floor(u), 0, len(tab) - 2).astype(np.int64)
    f = u - i
    return tab[i] + f * (tab[i + 1] - tab[i])


def ssb_delay(det, t: np.ndarray) -> np.ndarray:
    """Delta_X(t) = r(t).n/c of Eq. t-ssb-equation, from the detector's FP64 table."""
    return _lerp(det.eph_t0, det.eph_dt, det.ssb_delay, t)


def periapsis_time(tasc_rel: float, P: float, e: float, omega: float) -> float:
    """T_p from the time of ascension T_asc (relative to t0): at the ascending node the
    argument of latitude omega + nu vanishes, so the true anomaly there is -omega; its
    eccentric and mean anomalies (Eq. solve-for-E) fix T_p = T_asc - M_asc / Omega.
    For e = 0 this is T_asc + omega / Omega, and the orbit is the circular one."""
    nu = -omega
    E = 2.0 * math.atan2(math.sqrt(1.0 - e) * math.sin(0.5 * nu), math.sqrt(1.0 + e) * math.cos(0.5 * nu))
    M = E - e * math.sin(E)
    return tasc_rel - M * P / (2.0 * math.pi)


def kepler_E(M: np.ndarray, e: float) -> np.ndarray:
    """Eccentric anomaly: the root of E - e sin E = M (Eq. solve-for-E), by Newton's
    method from E = M + e sin M, to FP64 precision."""
    M = np.asarray(M, np.float64)
    E = M + e * np.sin(M)
    for _ in range(50):
        dE = (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
        E = E - dE
        if np.all(np.abs(dE) < 1e-15 * np.maximum(1.0, np.abs(E))):
            break
    return E


def binary_delay(a_p: float, tasc_rel: float, P: float, u: np.ndarray, e: float = 0.0,
                 omega: float = 0.0) -> np.ndarray:
    """R/c at SSB time u (relative to t0): a_p [sin w (cos E - e) + cos w sqrt(1 - e^2) sin E]
    (Eq. Kepler-equation) with E from the mean anomaly Omega (u - T_p) (Eq. solve-for-E;
    the anomaly taken at t_SSB as in reading 1).  e = 0: a_p sin(Omega (u - T_asc))."""
    u = np.asarray(u, np.float64)
    if e == 0.0:
        return a_p * np.sin(2.0 * np.pi * ((u - tasc_rel) / P))
    Tp = periapsis_time(tasc_rel, P, e, omega)
    E = kepler_E(2.0 * np.pi * ((u - Tp) / P), e)
    return a_p * (math.sin(omega) * (np.cos(E) - e) + math.cos(omega) * math.sqrt(1.0 - e * e) * np.sin(E))


def delay(det, a_p: float, tasc_rel: float, P: float, tau: np.ndarray, e: float = 0.0,
          omega: float = 0.0) -> np.ndarray:
    """d(tau) = tau - t(tau): detector time t whose source time tau(t) is tau.

    tau(t) = t_SSB - R(t_SSB)/c, t_SSB = t + Delta_X(t) (Eqs. t-ssb-equation,
    tau-equation; R/c the Roemer delay of binary_delay, circular for e = 0; reading 1:
    the orbital anomaly is taken at t_SSB, as Eq. tau-equation writes it).  Inversion by
    the two fixed points u = tau + R(u)/c and t = u - Delta_X(t), iterated on the small
    quantities b = u - tau and Delta = u - t so that d = Delta - b keeps FP64 precision
    (~1e-13 s).  All times are relative to t0.
    """
    tau = np.asarray(tau, np.float64)
    b = np.zeros_like(tau)
    for _ in range(N_FIXED_POINT):
        b = binary_delay(a_p, tasc_rel, P, tau + b, e, omega)
    dl = ssb_delay(det, tau)
    for _ in range(N_FIXED_POINT):
        dl = ssb_delay(det, (tau + b) - dl)
    return dl - b


def orbit(tmpl):
    """(a_p, T_asc, P, e, omega) of a template row; three-element rows are circular."""
    t = [float(v) for v in tmpl]
    return (t[0], t[1], t[2], t[3], t[4]) if len(t) >= 5 else (t[0], t[1], t[2], 0.0, 0.0)


# ---------------------------------------------------------------------------
# S2: windowed-sinc interpolation + heterodyne correction
#     (Eqs. shannon-interp-formula, delta-q-eq, q-prime-eq, resampled-time-series-q-eq)
# ---------------------------------------------------------------------------
def hamming(D: int) -> np.ndarray:
    """Hamming window of length 2D+1 on the tap index n = 0..2D (reading 2: the
    paper names the window but not its coefficients; w_D = 1 keeps integer
    points exact)."""
    n = np.arange(2 * D + 1, dtype=np.float64)
    return 0.54 - 0.46 * np.cos(2.0 * np.pi * n / (2 * D))


def stencil_position(e: np.ndarray, r: np.ndarray):
    """j* = round(t/dt') with ties rounded up (reading 3) and delta = t/dt' - j* in
    [-1/2, 1/2), for t/dt' = r - e (e = d/dt', r integer) (Eqs. delta-q-eq, q-prime-eq).
    Computed from the small quantity e so that delta keeps FP64 precision."""
    g = 0.5 - np.asarray(e, np.float64)
    fl = np.floor(g)
    jstar = np.asarray(r, np.int64) + fl.astype(np.int64)
    delta = (g - 0.5) - fl
    return jstar, delta


def interpolate(x: np.ndarray, jstar: np.ndarray, delta: np.ndarray, D: int) -> np.ndarray:
    """x(t) ~ sum_{j=j*-D}^{j*+D} x_j w_{j-j*+D} sinc(delta_j), delta_j = (t - t_j)/dt'.

    This is Eq. shannon-interp-formula with its alternating-sign form rewritten
    through sin(pi delta_j) = (-1)^(j-j0) sin(pi delta_j0); the sinc form returns
    x_{j*} exactly at delta = 0.  Samples outside [0, N_t) are zero."""
    x = np.asarray(x)
    N_t = x.shape[0]
    w = hamming(D)
    acc = np.zeros(np.shape(delta), np.complex128)
    for n in range(2 * D + 1):
        j = jstar - D + n
        ok = (j >= 0) & (j < N_t)
        xj = np.where(ok, x[np.clip(j, 0, N_t - 1)], 0.0)
        acc += xj * (w[n] * np.sinc(delta - (n - D)))
    return acc


def timing(det, cfg, plan: Plan, tmpl):
    """(j*, delta, d) for every source sample r = 0..M N_s - 1 of one detector and
    one template (a_p, T_asc, P)."""
    a_p, tasc, P, e, omega = orbit(tmpl)
    n = plan.M * plan.N_s
    r = np.arange(n, dtype=np.int64)
    d = delay(det, a_p, tasc - cfg.t0, P, r * plan.dt, e, omega)
    jstar, delta = stencil_position(d / plan.dt, r)
    return jstar, delta, d


def resample(x: np.ndarray, det, cfg, plan: Plan, tmpl, interp=None):
    """Source-frame series x'_r, r = 0..M N_s - 1, of one detector for one template:
    the interpolated x'(t(tau_r)) times exp(-2 pi i f_h [tau_r - t(tau_r)])
    (Eq. resampled-time-series-q-eq; reading 4: the printed exponent lacks the i
    that the sentence before it has).  Returns (x'_r, j*, delta).  `interp`, if
    given, replaces the windowed sinc: interp(x, j*, delta) -> x(t)."""
    jstar, delta, d = timing(det, cfg, plan, tmpl)
    xi = interpolate(x, jstar, delta, cfg.D) if interp is None else interp(x, jstar, delta)
    cyc = cfg.f_h * d
    cyc = cyc - np.floor(cyc)
    return xi * np.exp(-2j * np.pi * cyc), jstar, delta


# ---------------------------------------------------------------------------
# Antenna/noise weights (Eq. norm-a-eq and Sec. III B 1, III B 5)
# ---------------------------------------------------------------------------
def noise_block(jstar: np.ndarray, delta: np.ndarray, nsft: int) -> np.ndarray:
    """Index of the T_sft block holding detector time t = (j* + delta) dt':
    floor((j* + delta)/nsft), evaluated exactly from the integer j* and the sign
    of delta."""
    q = np.floor_divide(jstar, nsft)
    rem = jstar - q * nsft
    return np.where((rem == 0) & (delta < 0), q - 1, q)


def weights(det, cfg, jstar: np.ndarray, delta: np.ndarray):
    """alpha_r = a(t_r) m_r / sigma^2(t_r), beta_r = b(t_r) m_r / sigma^2(t_r) and
    sigma^2(t_r), at the detector time t_r = t(tau_r) the source sample was taken
    from (reading 5: inverse-variance weights, as a_r is proportional to a x / S_h;
    the paper resamples the per-SFT noise weights along with the data, so the gap
    mask and sigma follow the data; a, b vary over a sidereal day, so a(t_r) is
    the paper's a(r dt') up to a Roemer delay).  sigma is constant per T_sft block
    and m_r = 0 in gaps (sigma = 0), giving gaps zero weight in rho and in the
    normalisation (Sec. III B 1)."""
    nsft = int(round(cfg.T_sft / cfg.dt))
    t = (jstar + delta) * cfg.dt
    a = _lerp(det.ab_t0, det.ab_dt, det.a_tab, t)
    b = _lerp(det.ab_t0, det.ab_dt, det.b_tab, t)
    blk = noise_block(jstar, delta, nsft)
    ok = (blk >= 0) & (blk < len(det.sigma))
    sig = np.where(ok, det.sigma[np.clip(blk, 0, len(det.sigma) - 1)], 0.0)
    m = sig > 0
    s2 = np.where(m, sig * sig, 1.0)
    alpha = np.where(m, a / s2, 0.0)
    beta = np.where(m, b / s2, 0.0)
    return alpha, beta, np.where(m, sig * sig, 0.0)


# ---------------------------------------------------------------------------
# S3: per-segment spectra  (Eqs. fft-inklings ... F-bar definitions)
# ---------------------------------------------------------------------------
def spectra_direct(y: np.ndarray, plan: Plan) -> np.ndarray:
    """F_K(f_k) = sum_{r in segment K} y_r exp(-2 pi i (f_k - f_h)(tau_r - t0)),
    a direct DFT at the published frequencies; returns [M][N_f].  The common
    epoch t0 carries Phi_in (segment start) and makes Phi_out zero."""
    out = np.empty((plan.M, plan.N_f), np.complex128)
    for K in range(plan.M):
        r = np.arange(K * plan.N_s, (K + 1) * plan.N_s, dtype=np.float64)
        cyc = np.outer(plan.dfreq, r * plan.dt)
        cyc -= np.floor(cyc)
        out[K] = np.exp(-2j * np.pi * cyc) @ y[K * plan.N_s:(K + 1) * plan.N_s]
    return out


def spectra_fft(y: np.ndarray, plan: Plan) -> np.ndarray:
    """The same spectra through a zero-padded FP64 FFT of length N_FFT per segment:
    the segment is pre-rotated by exp(-2 pi i f_r* s dt'), transformed, the bin
    (k-bar - N_FFT/2) mod N_FFT is read (the FFT's lowest frequency f_FFT sits at
    k-bar = 0), and the segment-start phase exp(-2 pi i (f - f_h) K T_short) is
    applied (Phi_in)."""
    N = plan.N_FFT
    s = np.arange(plan.N_s, dtype=np.float64)
    pre = np.exp(-2j * np.pi * (plan.f_r * s * plan.dt))
    idx = np.mod(plan.kbar - N // 2, N)
    out = np.empty((plan.M, plan.N_f), np.complex128)
    for K in range(plan.M):
        seg = y[K * plan.N_s:(K + 1) * plan.N_s] * pre
        Y = np.fft.fft(seg, n=N)
        cyc = plan.dfreq * (K * plan.N_s * plan.dt)
        cyc = cyc - np.floor(cyc)
        out[K] = Y[idx] * np.exp(-2j * np.pi * cyc)
    return out


# ---------------------------------------------------------------------------
# S4: pairs and normalisation  (Sec. III B 1 pair selection; Eq. final-formatted-rho;
#     hat-A^2, hat-B^2, hat-C^2 of Appendix A)
# ---------------------------------------------------------------------------
def segment_norms(alpha, beta, s2, plan: Plan):
    """hat-A_XK = sum alpha^2 sigma^2, hat-B_XK = sum beta^2 sigma^2,
    hat-C_XK = sum alpha beta sigma^2 over segment K."""
    n = plan.M * plan.N_s
    A = (alpha[:n] ** 2 * s2[:n]).reshape(plan.M, plan.N_s).sum(axis=1)
    B = (beta[:n] ** 2 * s2[:n]).reshape(plan.M, plan.N_s).sum(axis=1)
    C = (alpha[:n] * beta[:n] * s2[:n]).reshape(plan.M, plan.N_s).sum(axis=1)
    return A, B, C


def pair_list(Q: int, M: int, R: int, mode: int) -> List[Tuple[int, int, int, int]]:
    """The pair set P as (X, K, Y, L) tuples.

    UNORDERED (reading 6): X < Y with |K - L| <= R (2R+1 partners, same-time
    cross-detector pairs included), and X = Y with 1 <= L - K <= R (R partners,
    auto-correlation excluded) -- each unordered pair once.
    CROSS_ONLY: the X < Y pairs alone.  ALL_ORDERED: every ordered pair with
    |K - L| <= R, auto-correlation included."""
    P = []
    for X in range(Q):
        for K in range(M):
            for Y in range(Q):
                for L in range(max(0, K - R), min(M, K + R + 1)):
                    if mode == PAIR_ALL_ORDERED:
                        P.append((X, K, Y, L))
                    elif X < Y:
                        P.append((X, K, Y, L))
                    elif X == Y and mode == PAIR_UNORDERED and 1 <= L - K:
                        P.append((X, K, Y, L))
    return P


def normalization(norms, plan: Plan, mode: int) -> float:
    """A^2_P + 2 C^2_P + B^2_P = sum over pairs of (A_K A_L + B_K B_L + 2 C_K C_L)."""
    Q = len(norms)
    tot = 0.0
    for (X, K, Y, L) in pair_list(Q, plan.M, plan.R, mode):
        A1, B1, C1 = norms[X][0][K], norms[X][1][K], norms[X][2][K]
        A2, B2, C2 = norms[Y][0][L], norms[Y][1][L], norms[Y][2][L]
        tot += A1 * A2 + B1 * B2 + 2.0 * C1 * C2
    return tot


def pair_sum(Fa, Fb, plan: Plan, mode: int) -> np.ndarray:
    """Re sum over pairs of conj(F_a,XK) F_a,YL + conj(F_b,XK) F_b,YL, per bin."""
    Q = len(Fa)
    acc = np.zeros(plan.N_f, np.float64)
    for (X, K, Y, L) in pair_list(Q, plan.M, plan.R, mode):
        acc += (np.conj(Fa[X][K]) * Fa[Y][L] + np.conj(Fb[X][K]) * Fb[Y][L]).real
    return acc


# ---------------------------------------------------------------------------
# Whole statistic
# ---------------------------------------------------------------------------
def rho_template(ds, tmpl, plan: Optional[Plan] = None, spectra: str = "fft",
                 mode: Optional[int] = None, return_parts: bool = False, interp=None):
    """rho_k for one template (Eq. final-formatted-rho): sqrt(2) times the pair sum
    over sqrt(A^2 + 2C^2 + B^2).  `interp` as in resample()."""
    cfg = ds.cfg
    plan = plan or make_plan(cfg)
    mode = cfg.pair_mode if mode is None else mode
    spec = spectra_fft if spectra == "fft" else spectra_direct
    Fa, Fb, norms = [], [], []
    for q, det in enumerate(ds.dets):
        xr, jstar, delta = resample(ds.x[q], det, cfg, plan, tmpl, interp)
        alpha, beta, s2 = weights(det, cfg, jstar, delta)
        Fa.append(spec(alpha * xr, plan))
        Fb.append(spec(beta * xr, plan))
        norms.append(segment_norms(alpha, beta, s2, plan))
    Dn = normalization(norms, plan, mode)
    raw = pair_sum(Fa, Fb, plan, mode)
    rho_k = math.sqrt(2.0) * raw / math.sqrt(Dn) if Dn > 0 else np.zeros_like(raw)
    if return_parts:
        return rho_k, dict(Fa=Fa, Fb=Fb, norms=norms, D=Dn, raw=raw, plan=plan)
    return rho_k


def rho(ds, templates=None, spectra: str = "fft", mode: Optional[int] = None,
        plan: Optional[Plan] = None, interp=None) -> np.ndarray:
    """rho[template][bin] for a set of templates."""
    plan = plan or make_plan(ds.cfg)
    tm = ds.templates if templates is None else np.asarray(templates, np.float64)
    return np.stack([rho_template(ds, t, plan, spectra, mode, interp=interp) for t in tm])


def topk(rho_tb: np.ndarray, k: int):
    """The k largest rho over (template, bin): descending rho, ties broken by
    (template, bin) ascending.  Returns (template, bin, rho) arrays."""
    flat = np.asarray(rho_tb, np.float64).ravel()
    order = np.lexsort((np.arange(flat.size), -flat))[:k]
    nb = rho_tb.shape[1]
    return order // nb, order % nb, flat[order]


# ---------------------------------------------------------------------------
# Detector-frame form (Eqs. from-here-resamp / well-formatted-rho): brute-force check
# ---------------------------------------------------------------------------
def detector_frame_rho(ds, tmpl, plan: Optional[Plan] = None, mode: Optional[int] = None):
    """rho from detector-frame samples without resampling: each raw sample j enters
    segment K by its source time tau(t_j), with phase 2 pi [(f - f_h) tau(t_j)
    + f_h (tau(t_j) - t_j)], its weights at t_j and the Jacobian d tau/dt -- the
    Riemann sum, over detector time, of the same integral the resampled sum takes
    over source time (Sec. III B 6: the resampled rho equals the detector-frame
    one when the Roemer delay is zero).  The normalisation is the resampled one.
    Tiny inputs only."""
    cfg = ds.cfg
    plan = plan or make_plan(cfg)
    mode = cfg.pair_mode if mode is None else mode
    a_p, tasc, P, e, _ = orbit(tmpl)
    tasc -= cfg.t0
    if e != 0.0:
        raise ValueError("the detector-frame brute force is written for circular orbits")
    Fa, Fb, norms = [], [], []
    for q, det in enumerate(ds.dets):
        _, jr, dr = resample(ds.x[q], det, cfg, plan, tmpl)
        norms.append(segment_norms(*weights(det, cfg, jr, dr), plan))
        j = np.arange(cfg.n_samples, dtype=np.int64)
        t = j * cfg.dt
        dl = ssb_delay(det, t)
        tssb = t + dl
        ph = 2.0 * np.pi * ((tssb - tasc) / P)
        tau = tssb - a_p * np.sin(ph)
        u = (t - det.eph_t0) / det.eph_dt
        i = np.clip(np.floor(u), 0, len(det.ssb_delay) - 2).astype(np.int64)
        ddl = (det.ssb_delay[i + 1] - det.ssb_delay[i]) / det.eph_dt
        jac = (1.0 + ddl) * (1.0 - a_p * (2.0 * np.pi / P) * np.cos(ph))
        alpha, beta, _ = weights(det, cfg, j, np.zeros(j.shape))
        K = np.floor(tau / (plan.N_s * plan.dt)).astype(np.int64)
        fa = np.zeros((plan.M, plan.N_f), np.complex128)
        fb = np.zeros((plan.M, plan.N_f), np.complex128)
        het = cfg.f_h * (tau - t)
        het -= np.floor(het)
        for KK in range(plan.M):
            sel = K == KK
            if not np.any(sel):
                continue
            cyc = np.outer(plan.dfreq, tau[sel]) + het[sel][None, :]
            cyc -= np.floor(cyc)
            v = ds.x[q][sel] * jac[sel]
            E = np.exp(-2j * np.pi * cyc)
            fa[KK] = E @ (v * alpha[sel])
            fb[KK] = E @ (v * beta[sel])
        Fa.append(fa)
        Fb.append(fb)
    Dn = normalization(norms, plan, mode)
    raw = pair_sum(Fa, Fb, plan, mode)
    return math.sqrt(2.0) * raw / math.sqrt(Dn)
