"""Seeded synthetic inputs shaped like the paper's Sco X-1 directed search.

This module generates *inputs* only: heterodyned complex detector series with
Gaussian noise, lock/unlock gaps and an optional injected CW signal, the
per-detector tables the method consumes (SSB delay, antenna functions a/b,
noise level per T_sft block) and the orbital template grid.  It holds none of
the resampled cross-correlation arithmetic (no timing inversion, no
interpolation, no FFT, no pair sum, no plan quantities); the oracle and the
CUDA path both take its output as given and share nothing else.

Physical set-up (Table I of the paper): Sco X-1 at
alpha = 16h19m55.067s, delta = -15d38m25.02s, P = 68023.70 s,
a_p ~ 1.44 lt-s, T_asc near the O1 epoch.  Detector motion uses a synthetic
ephemeris (circular 1-AU Earth orbit at the J2000 obliquity plus Earth
rotation) because no LAL ephemeris file is available; the antenna functions
a(t), b(t) are the Jaranowski-Krolak-Schutz closed forms for interferometers
with perpendicular arms at the H1/L1 sites.

Random numbers come from numpy's PCG64 with the seed given by the caller.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# Constants
# ---------------------------------------------------------------------------
AU_LIGHT_S = 499.004783836          # astronomical unit in light-seconds
R_EARTH_LIGHT_S = 6.371e6 / 299792458.0
OBLIQUITY = math.radians(23.4392911)
SIDEREAL_DAY = 86164.0905
SIDEREAL_YEAR = 365.256363004 * 86400.0

SCO_X1_ALPHA = math.radians((16 + 19 / 60 + 55.067 / 3600) * 15.0)
SCO_X1_DELTA = -math.radians(15 + 38 / 60 + 25.02 / 3600)
SCO_X1_P = 68023.70
T0_GPS = 1.1264e9                   # start of the synthetic observation
T_ASC_O1 = 1131415400.0             # inside the O1-epoch T_asc window of the paper


@dataclasses.dataclass(frozen=True)
class Site:
    name: str
    lat: float     # geodetic latitude [rad]
    lon: float     # east longitude [rad]
    gamma: float   # arm-bisector orientation, counter-clockwise from local East [rad]


H1 = Site("H1", math.radians(46.4551), math.radians(-119.4077), math.radians(171.8))
L1 = Site("L1", math.radians(30.5629), math.radians(-90.7742), math.radians(243.0))
SITES = (H1, L1)


def sky_unit_vector(alpha: float, delta: float) -> np.ndarray:
    return np.array([math.cos(alpha) * math.cos(delta),
                     math.sin(alpha) * math.cos(delta),
                     math.sin(delta)])


def _sidereal_angle(t_rel: np.ndarray, site: Site) -> np.ndarray:
    # Local sidereal angle; the Greenwich angle at the start is arbitrary but fixed.
    theta_g0 = math.radians(100.0)
    return theta_g0 + site.lon + 2.0 * math.pi * t_rel / SIDEREAL_DAY


def ssb_delay_analytic(site: Site, t_rel: np.ndarray,
                       alpha: float = SCO_X1_ALPHA, delta: float = SCO_X1_DELTA) -> np.ndarray:
    """Roemer delay r(t).n/c [s] of the detector relative to the SSB (synthetic ephemeris)."""
    n = sky_unit_vector(alpha, delta)
    lam = math.radians(350.0) + 2.0 * math.pi * np.asarray(t_rel, float) / SIDEREAL_YEAR
    ex = AU_LIGHT_S * np.cos(lam)
    ey = AU_LIGHT_S * np.sin(lam) * math.cos(OBLIQUITY)
    ez = AU_LIGHT_S * np.sin(lam) * math.sin(OBLIQUITY)
    th = _sidereal_angle(np.asarray(t_rel, float), site)
    sx = R_EARTH_LIGHT_S * math.cos(site.lat) * np.cos(th)
    sy = R_EARTH_LIGHT_S * math.cos(site.lat) * np.sin(th)
    sz = R_EARTH_LIGHT_S * math.sin(site.lat) * np.ones_like(th)
    return (ex + sx) * n[0] + (ey + sy) * n[1] + (ez + sz) * n[2]


def antenna_ab_analytic(site: Site, t_rel: np.ndarray,
                        alpha: float = SCO_X1_ALPHA, delta: float = SCO_X1_DELTA):
    """JKS amplitude modulation functions a(t), b(t) for perpendicular arms."""
    lam, g = site.lat, site.gamma
    h = alpha - _sidereal_angle(np.asarray(t_rel, float), site)    # hour angle, sign as JKS
    s2g, c2g = math.sin(2 * g), math.cos(2 * g)
    a = (s2g * (3 - math.cos(2 * lam)) * (3 - math.cos(2 * delta)) * np.cos(2 * h) / 16.0
         - c2g * math.sin(lam) * (3 - math.cos(2 * delta)) * np.sin(2 * h) / 4.0
         + s2g * math.sin(2 * lam) * math.sin(2 * delta) * np.cos(h) / 4.0
         - c2g * math.cos(lam) * math.sin(2 * delta) * np.sin(h) / 2.0
         + 0.75 * s2g * math.cos(lam) ** 2 * math.cos(delta) ** 2)
    b = (c2g * math.sin(lam) * math.sin(delta) * np.cos(2 * h)
         + s2g * (3 - math.cos(2 * lam)) * math.sin(delta) * np.sin(2 * h) / 4.0
         + c2g * math.cos(lam) * math.cos(delta) * np.cos(h)
         + s2g * math.sin(2 * lam) * math.cos(delta) * np.sin(h) / 2.0)
    return a, b


# ---------------------------------------------------------------------------
# Data containers
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class SearchConfig:
    """Search set-up: sampling, band and coherence parameters of one band."""
    t0: float                 # GPS time of sample 0 (detector frame) and of tau grid origin
    dt: float                 # sampling interval delta t' [s]
    n_samples: int            # samples per detector
    f_h: float                # heterodyne frequency = band centre [Hz]
    f_band: float             # searched band width [Hz]
    T_sft: float              # noise-estimation block length [s]
    T_max: float              # maximum lag [s]
    T_short: float = 0.0      # segment length; 0 means max(T_max, T_sft)
    mu_f: float = 0.1         # frequency mismatch
    D: int = 8                # Dirichlet terms of the windowed-sinc stencil (2D+1 taps)
    n_det: int = 2
    pair_mode: int = 0        # 0 unordered (default), 1 cross-detector only, 2 all ordered incl. auto


@dataclasses.dataclass
class DetectorTables:
    """Per-detector inputs; all times are relative to SearchConfig.t0."""
    name: str
    eph_t0: float             # time of ssb_delay[0]
    eph_dt: float
    ssb_delay: np.ndarray     # float64, t_SSB - t at eph_t0 + n*eph_dt
    ab_t0: float              # time of a_tab[0]
    ab_dt: float
    a_tab: np.ndarray         # float64
    b_tab: np.ndarray         # float64
    sigma: np.ndarray         # float64 noise std per T_sft block starting at 0; 0 marks a gap


@dataclasses.dataclass
class Injection:
    h0: float
    f0: float
    a_p: float
    T_asc: float              # GPS
    P: float
    cosi: float = 1.0
    psi: float = 0.0
    phi0: float = 0.0
    e: float = 0.0            # eccentricity (0: circular orbit)
    omega: float = 0.0        # argument of periapsis [rad]


@dataclasses.dataclass
class Dataset:
    cfg: SearchConfig
    dets: List[DetectorTables]
    x: np.ndarray             # complex128 [Q][N_t] heterodyned series (zero in gaps)
    templates: np.ndarray     # float64 [T][3] = (a_p [lt-s], T_asc [GPS s], P [s])
    injection: Optional[Injection] = None
    description: str = ""

    @property
    def x64(self) -> np.ndarray:
        return np.ascontiguousarray(self.x.astype(np.complex64))


# ---------------------------------------------------------------------------
# Generators
# ---------------------------------------------------------------------------
def lock_mask(n_blocks: int, duty: float, mean_lock_blocks: float,
              rng: np.random.Generator) -> np.ndarray:
    """Lock (True) / unlock (False) state per block: a two-state Markov chain whose
    lock and unlock durations are geometric (discrete exponential) with the mean lock
    length given and the mean unlock length set so the duty cycle is `duty`."""
    if duty >= 1.0:
        return np.ones(n_blocks, bool)
    mean_unlock = max(mean_lock_blocks * (1.0 - duty) / duty, 1.0)
    p_lose, p_regain = 1.0 / mean_lock_blocks, 1.0 / mean_unlock
    out = np.empty(n_blocks, bool)
    state = rng.random() < duty
    u = rng.random(n_blocks)
    for i in range(n_blocks):
        out[i] = state
        state = (u[i] >= p_lose) if state else (u[i] < p_regain)
    return out


def make_detector_tables(site: Site, cfg: SearchConfig, sigma_blocks: np.ndarray,
                         eph_dt: float = 8.0, ab_dt: float = 60.0,
                         zero_roemer: bool = False, const_ab: Optional[Sequence[float]] = None,
                         ) -> DetectorTables:
    T_obs = cfg.n_samples * cfg.dt
    pad = 2048.0
    eph_t0 = -pad
    n_eph = int(math.ceil((T_obs + 2 * pad) / eph_dt)) + 1
    t_eph = eph_t0 + eph_dt * np.arange(n_eph)
    ssb = np.zeros(n_eph) if zero_roemer else ssb_delay_analytic(site, t_eph)
    n_ab = int(math.ceil(T_obs / ab_dt)) + 2
    t_ab = ab_dt * np.arange(n_ab)
    if const_ab is not None:
        a_tab = np.full(n_ab, float(const_ab[0]))
        b_tab = np.full(n_ab, float(const_ab[1]))
    else:
        a_tab, b_tab = antenna_ab_analytic(site, t_ab)
    return DetectorTables(site.name, eph_t0, eph_dt, ssb, 0.0, ab_dt, a_tab, b_tab,
                          np.asarray(sigma_blocks, float))


def _table_lerp(t0: float, dt: float, tab: np.ndarray, t: np.ndarray) -> np.ndarray:
    u = (t - t0) / dt
    i = np.clip(np.floor(u).astype(np.int64), 0, len(tab) - 2)
    f = u - i
    return tab[i] * (1.0 - f) + tab[i + 1] * f


def orbital_roemer_delay(inj: Injection, tasc_rel: float, tssb: np.ndarray) -> np.ndarray:
    """R/c of the injected orbit at SSB times tssb (relative to t0): circular,
    a_p sin(2 pi (tssb - T_asc)/P), or Keplerian with eccentricity e and argument of
    periapsis omega, the periapsis time placed so the ascending node (true anomaly
    -omega) is at T_asc; Kepler's equation solved by bisection."""
    if inj.e == 0.0:
        return inj.a_p * np.sin(2.0 * np.pi * ((tssb - tasc_rel) / inj.P))
    e, w = inj.e, inj.omega
    nu = -w
    E_asc = 2.0 * math.atan(math.sqrt((1.0 - e) / (1.0 + e)) * math.tan(0.5 * nu))
    tp = tasc_rel - (E_asc - e * math.sin(E_asc)) * inj.P / (2.0 * math.pi)
    M = 2.0 * np.pi * ((tssb - tp) / inj.P)
    M = M - 2.0 * np.pi * np.floor(M / (2.0 * np.pi))              # [0, 2 pi)
    lo, hi = np.zeros_like(M), np.full_like(M, 2.0 * np.pi)         # E - e sin E is increasing
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = mid - e * np.sin(mid) < M
        lo, hi = np.where(below, mid, lo), np.where(below, hi, mid)
    E = 0.5 * (lo + hi)
    return inj.a_p * (math.sin(w) * (np.cos(E) - e) + math.cos(w) * math.sqrt(1.0 - e * e) * np.sin(E))


def inject_signal(inj: Injection, cfg: SearchConfig, site: Site, det: DetectorTables,
                  exact_ephemeris: bool = True, exact_antenna: bool = True) -> np.ndarray:
    """Heterodyned complex CW signal at the detector sample times.

    s(t) = 1/2 h0 [F+ A+ - i Fx Ax] exp(i Phi(t)), with the phase model of the
    paper's signal model, Phi = phi0 + 2 pi f0 (tau(t) - t0),
    tau = t_SSB - a_p sin(2 pi (t_SSB - T_asc)/P), t_SSB = t + r.n/c, and
    heterodyned by exp(-2 pi i f_h (t - t0)).  Phase is accumulated in cycles
    relative to t0 to keep FP64 precision.
    """
    t = cfg.dt * np.arange(cfg.n_samples, dtype=np.float64)
    if exact_ephemeris:
        delay = (np.zeros_like(t) if not np.any(det.ssb_delay) else ssb_delay_analytic(site, t))
    else:
        delay = _table_lerp(det.eph_t0, det.eph_dt, det.ssb_delay, t)
    tasc_rel = inj.T_asc - cfg.t0
    tssb = t + delay
    binary = orbital_roemer_delay(inj, tasc_rel, tssb)
    # f0 (tau - t0) - f_h (t - t0) = f0 (delay - binary) + (f0 - f_h) t
    cyc = inj.f0 * (delay - binary)
    cyc = cyc - np.floor(cyc)
    cyc2 = (inj.f0 - cfg.f_h) * t
    cyc2 = cyc2 - np.floor(cyc2)
    phase = 2.0 * np.pi * (cyc + cyc2) + inj.phi0
    if exact_antenna and np.ptp(det.a_tab) > 0:
        a, b = antenna_ab_analytic(site, t)
    else:
        a = _table_lerp(det.ab_t0, det.ab_dt, det.a_tab, t)
        b = _table_lerp(det.ab_t0, det.ab_dt, det.b_tab, t)
    c2p, s2p = math.cos(2 * inj.psi), math.sin(2 * inj.psi)
    Fp = a * c2p + b * s2p
    Fx = b * c2p - a * s2p
    Ap = 0.5 * (1.0 + inj.cosi ** 2)
    Ax = inj.cosi
    return 0.5 * inj.h0 * (Fp * Ap - 1j * Fx * Ax) * np.exp(1j * phase)


def build_dataset(cfg: SearchConfig, templates: np.ndarray, seed: int,
                  duty: float = 1.0, mean_lock_s: float = 6 * 3600.0,
                  injection: Optional[Injection] = None, noise: bool = True,
                  sigma_jitter: float = 0.0, zero_roemer: bool = False,
                  const_ab: Optional[Sequence[float]] = None, eph_dt: float = 8.0,
                  ab_dt: float = 60.0, description: str = "") -> Dataset:
    rng = np.random.default_rng(seed)
    T_obs = cfg.n_samples * cfg.dt
    n_blocks = int(math.ceil(T_obs / cfg.T_sft))
    nsft = int(round(cfg.T_sft / cfg.dt))
    dets, xs = [], []
    for q in range(cfg.n_det):
        site = SITES[q % len(SITES)]
        lock = lock_mask(n_blocks, duty, mean_lock_s / cfg.T_sft, rng)
        sig = np.ones(n_blocks)
        if sigma_jitter > 0:
            sig = 1.0 + sigma_jitter * (2.0 * rng.random(n_blocks) - 1.0)
        sig = np.where(lock, sig, 0.0)
        det = make_detector_tables(site, cfg, sig, eph_dt=eph_dt, ab_dt=ab_dt,
                                   zero_roemer=zero_roemer, const_ab=const_ab)
        sig_samp = np.repeat(sig, nsft)[: cfg.n_samples]
        x = np.zeros(cfg.n_samples, np.complex128)
        if noise:
            re = rng.standard_normal(cfg.n_samples)
            im = rng.standard_normal(cfg.n_samples)
            x += (re + 1j * im) * (sig_samp / math.sqrt(2.0))
        if injection is not None:
            x += inject_signal(injection, cfg, site, det,
                               exact_ephemeris=not zero_roemer,
                               exact_antenna=const_ab is None)
        x[sig_samp == 0.0] = 0.0
        dets.append(det)
        xs.append(x)
    return Dataset(cfg, dets, np.stack(xs), np.ascontiguousarray(templates, dtype=np.float64),
                   injection, description)


def template_grid(a_p: Sequence[float], T_asc: Sequence[float], P: Sequence[float]) -> np.ndarray:
    A, T, PP = np.meshgrid(np.asarray(a_p, float), np.asarray(T_asc, float),
                           np.asarray(P, float), indexing="ij")
    return np.stack([A.ravel(), T.ravel(), PP.ravel()], axis=1)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
def plain_day(seed: int = 1001, loudness: float = 1.0, noise: bool = True,
              f0: Optional[float] = None, D: int = 8) -> Dataset:
    """One day, 1 Hz band at 100 Hz sampled at 1 Hz, 20% gaps, T_sft = 240 s,
    T_max = 0, 4x4x4 orbital grid with the injection on a node."""
    cfg = SearchConfig(t0=T0_GPS, dt=1.0, n_samples=86400, f_h=100.0, f_band=1.0,
                       T_sft=240.0, T_max=0.0, D=D)
    rng = np.random.default_rng(seed + 7)
    tasc = T_ASC_O1 + rng.uniform(-100.0, 100.0)
    inj = Injection(h0=0.05 * math.sqrt(2.0) * loudness,
                    f0=cfg.f_h + 0.1 if f0 is None else f0,
                    a_p=1.44, T_asc=tasc, P=SCO_X1_P, cosi=0.6, psi=0.3, phi0=0.7)
    tm = template_grid([1.40, 1.42, 1.44, 1.46], tasc + np.array([-40.0, 0.0, 40.0, 80.0]),
                       SCO_X1_P + np.array([-0.04, 0.0, 0.04, 0.08]))
    return build_dataset(cfg, tm, seed, duty=0.8, injection=inj, noise=noise,
                         description="1 day, 1 Hz band at 100 Hz, T_max=0, 64 templates")


def o1_band(seed: int = 1002, T_max: float = 3600.0, n_ap: int = 40, n_tasc: int = 200,
            days: float = 120.0, noise: bool = True, loudness: float = 1.0,
            f0: Optional[float] = None) -> Dataset:
    """120 days at 60% duty, 0.5 Hz band at 150 Hz sampled at 1 Hz, T_sft = 360 s,
    T_max = T_short = 3600 s, grid a_p in [1.36, 1.52] (n_ap) x T_asc +/- 300 s (n_tasc),
    P fixed.  With T_max = 36000 s this is the long-lag precision variant."""
    n = int(round(days * 86400.0))
    cfg = SearchConfig(t0=T0_GPS, dt=1.0, n_samples=n, f_h=150.0, f_band=0.5,
                       T_sft=360.0, T_max=T_max, T_short=T_max)
    rng = np.random.default_rng(seed + 7)
    tasc = T_ASC_O1 + rng.uniform(-100.0, 100.0)
    inj = Injection(h0=0.05 * math.sqrt(2.0) * loudness,
                    f0=cfg.f_h + 0.0731 if f0 is None else f0,
                    a_p=1.44, T_asc=tasc, P=SCO_X1_P, cosi=0.6, psi=0.3, phi0=0.7)
    tm = template_grid(np.linspace(1.36, 1.52, n_ap), tasc + np.linspace(-300.0, 300.0, n_tasc),
                       [SCO_X1_P])
    return build_dataset(cfg, tm, seed, duty=0.6, injection=inj, noise=noise,
                         description=f"{days:g} d, 0.5 Hz at 150 Hz, T_max={T_max:g} s, "
                                     f"{n_ap}x{n_tasc} templates")


def multiband_band(b: int, seed: int = 1003, n_bands: int = 32, days: float = 10.0,
                   template_scale: float = 1.0, noise: bool = True,
                   max_templates: Optional[int] = None) -> Dataset:
    """Band b of the batched multi-band workload: 0.5 Hz at f0_b = 20 + 230 b/31 Hz
    sampled at 1 s, T_sft = T_short = T_max = 60 round(4 * 15^(b/31)) s (240 s at 20 Hz
    to 3600 s at 250 Hz), N_b = round(1e3 * 50^(b/31)) templates (about 4.2e5 over the
    32 bands) times template_scale, on an a_p x T_asc grid; T_obs = 10 d at 60 % duty
    with each band's gaps drawn from its own seed; an injection 0.0731 Hz above f0_b."""
    x = b / (n_bands - 1)
    f0 = 20.0 + 230.0 * x
    T = 60.0 * round(4.0 * 15.0 ** x)
    n_b = max(1, int(round(1e3 * 50.0 ** x * template_scale)))
    if max_templates is not None:
        n_b = min(n_b, max_templates)
    cfg = SearchConfig(t0=T0_GPS, dt=1.0, n_samples=int(round(days * 86400.0)), f_h=f0, f_band=0.5,
                       T_sft=T, T_max=T, T_short=T)
    rng = np.random.default_rng(seed + 101 * b)
    tasc = T_ASC_O1 + rng.uniform(-100.0, 100.0)
    inj = Injection(h0=0.1, f0=f0 + 0.0731, a_p=1.44, T_asc=tasc, P=SCO_X1_P, cosi=0.6, psi=0.3, phi0=0.7)
    n_ap = max(1, int(round(math.sqrt(n_b / 5.0))))
    n_tasc = max(1, int(round(n_b / n_ap)))
    tm = template_grid(np.linspace(1.36, 1.52, n_ap), tasc + np.linspace(-300.0, 300.0, n_tasc), [SCO_X1_P])
    tm = tm[:n_b] if len(tm) >= n_b else tm
    return build_dataset(cfg, tm, seed + 101 * b, duty=0.6, injection=inj, noise=noise,
                         description=f"band {b}: 0.5 Hz at {f0:.1f} Hz, T_max={T:g} s, {len(tm)} templates")


def multiband(seed: int = 1003, n_bands: int = 32, days: float = 10.0, template_scale: float = 1.0,
              bands: Optional[Sequence[int]] = None, noise: bool = True,
              max_templates: Optional[int] = None) -> List[Dataset]:
    """The batched multi-band workload: one Dataset per band (see multiband_band)."""
    idx = range(n_bands) if bands is None else bands
    return [multiband_band(b, seed, n_bands, days, template_scale, noise, max_templates) for b in idx]


def tiny(seed: int = 7, n_samples: int = 4096, T_sft: float = 64.0, T_max: float = 128.0,
         T_short: float = 128.0, f_h: float = 120.0, f_band: float = 0.5, D: int = 8,
         n_templates: int = 4, duty: float = 0.85, noise: bool = True,
         injection: Optional[Injection] = None, zero_roemer: bool = False,
         const_ab: Optional[Sequence[float]] = None, sigma_jitter: float = 0.2,
         pair_mode: int = 0, n_det: int = 2, mean_lock_s: float = 600.0,
         eph_dt: float = 8.0, ab_dt: float = 16.0, templates: Optional[np.ndarray] = None
         ) -> Dataset:
    """Small test workload: a few thousand samples and a handful of templates."""
    cfg = SearchConfig(t0=T0_GPS, dt=1.0, n_samples=n_samples, f_h=f_h, f_band=f_band,
                       T_sft=T_sft, T_max=T_max, T_short=T_short, D=D, n_det=n_det,
                       pair_mode=pair_mode)
    if templates is None:
        rng = np.random.default_rng(seed + 11)
        tasc = T_ASC_O1 + rng.uniform(-100.0, 100.0)
        templates = np.stack([rng.uniform(1.3, 1.6, n_templates),
                              tasc + rng.uniform(-300, 300, n_templates),
                              SCO_X1_P + rng.uniform(-0.1, 0.1, n_templates)], axis=1)
    return build_dataset(cfg, templates, seed, duty=duty, mean_lock_s=mean_lock_s,
                         injection=injection, noise=noise, sigma_jitter=sigma_jitter,
                         zero_roemer=zero_roemer, const_ab=const_ab, eph_dt=eph_dt,
                         ab_dt=ab_dt, description="tiny test workload")
