"""Plain FP64 NumPy restatement of the detector-frame ("demodulation") CrossCorr statistic.

TEST INFRASTRUCTURE: imported only by tests/ and the CPU legs of bench.py.

This is the statistic the paper's resampled method replaces (Sec. II, following
Whelan et al. 2015): data in short Fourier transforms, the signal's bins selected and
weighted by a sinc (Dirichlet) kernel per SFT, SFT pairs within T_max weighted by the
geometric filter and phased by the signal model.  Notation as the paper's:

* SFT K = (detector X, T_sft block k) over the locked blocks; mid-time t_K;
  x~_Km = sum_j x_K(t_K - T_sft/2 + j dt) exp(-2 pi i j m dt / T_sft) dt
  (Eq. fourier-transform-def), heterodyned bin m <-> frequency f_h + m/T_sft;
* z_Km = x~_Km sqrt(2 / (T_sft S_K)) with S_K = 2 sigma_K^2 dt, the one-sided PSD of
  complex white noise of variance sigma_K^2 per sample (Eq. normalized-z-bin), so that
  E|z_Km|^2 = 1;
* f_K = f dtau/dt(t_K), kappa_Km = m - (f_K - f_h) T_sft for the n_bin bins nearest the
  signal, Xi_K = sqrt(sum sinc^2 kappa), z_K = (1/Xi_K) sum (-1)^m sinc(kappa_Km) z_Km
  (Eq. total-data-eq);
* Gamma_KL = (a^_K a^_L + b^_K b^_L)/10 with a^_K = sqrt(2 T_sft/S_K) a(t_K)
  (Eq. geometric-filter);
* Phi_K = 2 pi (f tau(t_K) - f_h t_K), the heterodyned signal phase at t_K, and
  rho = N sum_{KL in P} Gamma_KL Xi_K Xi_L (exp(i (Phi_K - Phi_L)) z_K* z_L + c.c.),
  N = (2 sum_P Xi_K^2 Xi_L^2 Gamma_KL^2)^(-1/2) (Eqs. textbook-cc-rho, norm-cc).

Readings (numbered D1...):
D1. The paper prints both the 1/Xi_K of Eq. total-data-eq and the Xi_K^2 Xi_L^2 of
    Eq. norm-cc; they are consistent (Var rho = 1, the role of N) when each pair is also
    weighted by Xi_K Xi_L, which is also the optimal weight for a signal whose z_K grows
    as Xi_K.  That weight is taken.
D2. The pair set is every unordered pair of distinct SFTs with |t_K - t_L| <= T_max
    (the "+ c.c." form is symmetric, so an ordered double sum would count each twice):
    same-time pairs of different detectors and different-time pairs of any detectors.
D3. With n_bin = 2 the bins are floor(x) and floor(x) + 1 for x = (f_K - f_h) T_sft; in
    general the n_bin bins centred on x.
D4. a, b, sigma are taken at the SFT mid-time / per SFT block.
"""
from __future__ import annotations

import math
from typing import List, Optional

import numpy as np

from .crosscorr import kepler_E, make_plan, orbit, periapsis_time, ssb_delay


def sfts(ds):
    """Per detector: (block indices k, mid-times t_K, z_Km [n_sft, N] with bins in numpy
    FFT order, sigma_K) over the locked T_sft blocks (Eqs. fourier-transform-def,
    normalized-z-bin)."""
    cfg = ds.cfg
    N = int(round(cfg.T_sft / cfg.dt))
    out = []
    for q, det in enumerate(ds.dets):
        n_blk = min(len(det.sigma), cfg.n_samples // N)
        ks = np.array([k for k in range(n_blk) if det.sigma[k] > 0], np.int64)
        x = np.asarray(ds.x[q], np.complex128)
        seg = x[(ks[:, None] * N + np.arange(N)[None, :])] if len(ks) else np.zeros((0, N), np.complex128)
        xt = np.fft.fft(seg, axis=1) * cfg.dt                       # sum_j x_j exp(-2 pi i j m / N) dt
        sig = det.sigma[ks]
        S = 2.0 * sig * sig * cfg.dt
        z = xt * np.sqrt(2.0 / (cfg.T_sft * S))[:, None]
        tmid = (ks * N + 0.5 * N) * cfg.dt
        out.append((ks, tmid, z, sig))
    return out


def source_time(det, a_p: float, tasc_rel: float, P: float, t: np.ndarray, e: float = 0.0, omega: float = 0.0):
    """tau(t) - t = Delta_X(t) - R(t_SSB)/c and dtau/dt at detector times t (relative to
    t0; Eqs. t-ssb-equation, tau-equation, Kepler-equation with the anomaly at t_SSB):
    dtau/dt = (1 + Delta') (1 - dR/du / c), dE/du = Omega / (1 - e cos E)."""
    t = np.asarray(t, np.float64)
    dl = ssb_delay(det, t)
    u = t + dl
    u_i = (t - det.eph_t0) / det.eph_dt
    i = np.clip(np.floor(u_i), 0, len(det.ssb_delay) - 2).astype(np.int64)
    ddl = (det.ssb_delay[i + 1] - det.ssb_delay[i]) / det.eph_dt
    Om = 2.0 * np.pi / P
    if e == 0.0:
        ph = Om * (u - tasc_rel)
        R, dR = a_p * np.sin(ph), a_p * Om * np.cos(ph)
    else:
        Tp = periapsis_time(tasc_rel, P, e, omega)
        E = kepler_E(Om * (u - Tp), e)
        q = math.sqrt(1.0 - e * e)
        R = a_p * (math.sin(omega) * (np.cos(E) - e) + math.cos(omega) * q * np.sin(E))
        dR = a_p * (-math.sin(omega) * np.sin(E) + math.cos(omega) * q * np.cos(E)) * Om / (1.0 - e * np.cos(E))
    return dl - R, (1.0 + ddl) * (1.0 - dR)


def signal_bins(det, cfg, a_p: float, tasc_rel: float, P: float, tmid: np.ndarray, f: np.ndarray,
                e: float = 0.0, omega: float = 0.0):
    """(x, cyc): the signal's heterodyned bin position x = (f_K - f_h) T_sft with
    f_K = f dtau/dt(t_K), and its heterodyned phase in cycles, f tau(t_K) - f_h t_K
    reduced mod 1, for SFT mid-times t_K [n_sft] and frequencies f [n_f]."""
    d, dtau = source_time(det, a_p, tasc_rel, P, tmid, e, omega)
    dfreq = np.asarray(f, np.float64) - cfg.f_h
    # f tau - f_h t = f (tau - t) + (f - f_h) t, and its time derivative
    x = (np.outer(dtau - 1.0, f) + dfreq[None, :]) * cfg.T_sft
    cyc = np.outer(d, f) + np.outer(tmid, dfreq)
    return x, cyc - np.floor(cyc)


def _lerp(t0, dt, tab, t):
    u = (np.asarray(t, np.float64) - t0) / dt
    i = np.clip(np.floor(u), 0, len(tab) - 2).astype(np.int64)
    f = u - i
    return tab[i] + f * (tab[i + 1] - tab[i])


def sft_data_vector(z: np.ndarray, x: np.ndarray, n_bin: int = 2):
    """z_K and Xi_K (Eq. total-data-eq) for SFT bins z [n_sft, N] (numpy FFT order) and
    signal bin positions x = (f_K - f_h) T_sft, [n_sft, n_f]."""
    N = z.shape[1]
    m0 = np.floor(x).astype(np.int64) - (n_bin // 2 - 1)
    zK = np.zeros(x.shape, np.complex128)
    xi2 = np.zeros(x.shape, np.float64)
    rows = np.arange(z.shape[0])[:, None]
    for j in range(n_bin):
        m = m0 + j
        s = np.sinc(m - x)
        sign = np.where(m % 2 == 0, 1.0, -1.0)
        zK += sign * s * z[rows, m % N]
        xi2 += s * s
    xi = np.sqrt(xi2)
    return zK / xi, xi


def demod_rho(ds, tmpl, freqs: Optional[np.ndarray] = None, n_bin: int = 2, T_max: Optional[float] = None,
              sft_list=None):
    """rho(f) of one template (a_p, T_asc, P) at the frequencies `freqs` (default: the
    resampled plan's output frequencies), Eq. textbook-cc-rho with reading D1."""
    cfg = ds.cfg
    plan = make_plan(cfg)
    if freqs is None:
        dfreq = plan.dfreq
    else:
        dfreq = np.asarray(freqs, np.float64) - cfg.f_h
    f = cfg.f_h + dfreq
    T_max = cfg.T_max if T_max is None else T_max
    a_p, tasc, P, e, omega = orbit(tmpl)
    tasc_rel = tasc - cfg.t0
    sft_list = sfts(ds) if sft_list is None else sft_list
    T, Y, AH, BH, XI, DET = [], [], [], [], [], []
    for q, (det, (ks, tmid, z, sig)) in enumerate(zip(ds.dets, sft_list)):
        if len(ks) == 0:
            continue
        x, cyc = signal_bins(det, cfg, a_p, tasc_rel, P, tmid, f, e, omega)
        zK, xi = sft_data_vector(z, x, n_bin)
        Y.append(xi * zK * np.exp(-2j * np.pi * cyc))      # Xi_K z_K exp(-i Phi_K)
        XI.append(xi)
        S = 2.0 * sig * sig * cfg.dt
        scale = np.sqrt(2.0 * cfg.T_sft / S)
        AH.append(scale * _lerp(det.ab_t0, det.ab_dt, det.a_tab, tmid))
        BH.append(scale * _lerp(det.ab_t0, det.ab_dt, det.b_tab, tmid))
        T.append(tmid)
        DET.append(np.full(len(ks), q))
    if not T:
        return np.zeros(len(f))
    T, DET = np.concatenate(T), np.concatenate(DET)
    Y, XI = np.concatenate(Y), np.concatenate(XI)
    AH, BH = np.concatenate(AH), np.concatenate(BH)
    raw = np.zeros(len(f))
    den = np.zeros(len(f))
    order = np.argsort(T, kind="stable")        # each unordered pair once, visited in time order
    T, Y, XI, AH, BH = T[order], Y[order], XI[order], AH[order], BH[order]
    n = len(T)
    for K in range(n):
        for L in range(K + 1, n):
            if T[L] - T[K] > T_max + 1e-9:
                break
            g = (AH[K] * AH[L] + BH[K] * BH[L]) / 10.0
            # Xi_K Xi_L (e^{i(Phi_K - Phi_L)} z_K* z_L + c.c.) = 2 Re(conj(Y_K) Y_L)
            raw += g * 2.0 * np.real(np.conj(Y[K]) * Y[L])
            den += (XI[K] * XI[L] * g) ** 2
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(den > 0, raw / np.sqrt(2.0 * den), 0.0)


def pair_list(ds, T_max: Optional[float] = None, sft_list=None) -> List[tuple]:
    """The SFT pairs (X, k, Y, l) of reading D2, for the brute-force pin."""
    cfg = ds.cfg
    T_max = cfg.T_max if T_max is None else T_max
    sft_list = sfts(ds) if sft_list is None else sft_list
    items = [(tm, q, k) for q, (ks, tmid, _, _) in enumerate(sft_list) for k, tm in zip(ks, tmid)]
    out = []
    for i in range(len(items)):
        for j in range(i + 1, len(items)):
            if abs(items[i][0] - items[j][0]) <= T_max + 1e-9:
                out.append((items[i][1], int(items[i][2]), items[j][1], int(items[j][2])))
    return out
