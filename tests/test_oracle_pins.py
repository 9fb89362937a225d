"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle by a route other than retyping its formulas:
values the paper prints, closed forms, invariants, special cases and brute
force.  A plausible mistake anywhere in the oracle (a dropped term, a sign,
an index, a transposed operand) fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from synth import Dataset, Injection, SearchConfig

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _flat_dataset(cfg, x, sigma=None, a=1.0, b=0.0, templates=None):
    """Dataset with zero Roemer delay, constant antenna functions and given series."""
    dets = []
    nblk = int(math.ceil(cfg.n_samples * cfg.dt / cfg.T_sft))
    for q in range(cfg.n_det):
        sig = np.ones(nblk) if sigma is None else sigma[q]
        dets.append(synth.make_detector_tables(synth.SITES[q], cfg, sig, zero_roemer=True,
                                               const_ab=(a, b)))
    if templates is None:
        templates = np.array([[0.0, synth.T_ASC_O1, synth.SCO_X1_P]])
    return Dataset(cfg, dets, np.asarray(x, np.complex128), templates)


# ---------------------------------------------------------------------------
# Plan (Sec. III B 3-4)
# ---------------------------------------------------------------------------
def test_plan_printed_values():
    g = _golden("paper_printed_values.json")
    # mu_f = 0.1 makes the FFT duration at least 2.3 T_coh
    cfg = SearchConfig(t0=0.0, dt=1.0, n_samples=86400, f_h=100.0, f_band=1.0, T_sft=240.0,
                       T_max=240.0, T_short=240.0, mu_f=0.1)
    p = oracle.make_plan(cfg)
    assert round(1.0 / (p.dlf * p.T_coh), 1) == g["fft_duration_over_tcoh_at_mu_0.1"]["value"]
    # delta-lambda_f T_coh < 1 up to mu_f ~ 0.52
    mu_edge = g["mu_f_where_dlf_tcoh_reaches_1"]["value"]
    for mu, below in ((mu_edge - 0.005, True), (mu_edge + 0.01, False)):
        cfg.mu_f = mu
        q = oracle.make_plan(cfg)
        assert (q.dlf * q.T_coh < 1.0) == below


@pytest.mark.parametrize("f_band,T_max,f_h", [(1.0, 0.0, 100.0), (0.5, 3600.0, 150.0),
                                             (0.05, 3600.0, 150.0), (0.05, 720.0, 77.3),
                                             (0.3, 1080.0, 200.0)])
def test_plan_lowest_frequency_on_bin_k0(f_band, T_max, f_h):
    """The paper places the smallest output frequency f_h - f_band/2 on bin k0;
    this pins the readings of remainder(), f_FFT and lround (readings 7-9)."""
    cfg = SearchConfig(t0=0.0, dt=1.0, n_samples=200000, f_h=f_h, f_band=f_band,
                       T_sft=240.0, T_max=T_max)
    p = oracle.make_plan(cfg)
    assert abs(p.freq[0] - (f_h - f_band / 2)) < 1e-9
    assert np.all(np.diff(p.freq) > 0)
    assert p.freq[-1] < f_h + f_band / 2
    # N_FFT: the power of two at or above N_FFT0; decimation ratio >= 1
    assert p.N_FFT >= p.N_FFT0 > p.N_FFT / 2 and (p.N_FFT & (p.N_FFT - 1)) == 0
    assert p.nu_R >= 1.0
    # mean output spacing is the metric spacing delta-lambda_f
    assert abs((p.freq[-1] - p.freq[0]) / (p.N_f - 1) - p.dlf) < 1.0 / p.T_FFT / p.N_f * 2
    # |f_r*| is less than one FFT bin and f_FFT is the bottom of the Nyquist band
    assert abs(p.f_r) < 1.0 / p.T_FFT
    assert 0 <= p.k0 < p.N_FFT
    # decimation rounds down: each output frequency is at or below the ideal metric
    # grid point f_min + k delta-lambda_f, by less than one FFT bin
    ideal = (f_h - f_band / 2) + np.arange(p.N_f) * p.dlf
    gap = ideal - p.freq
    assert np.all(gap > -1e-9) and np.all(gap < 1.0 / p.T_FFT)


# ---------------------------------------------------------------------------
# Interpolation (Eq. shannon-interp-formula)
# ---------------------------------------------------------------------------
def test_interpolation_exact_at_integer_points():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(500) + 1j * rng.standard_normal(500)
    r = np.arange(20, 480)
    for shift in (-7, 0, 3):
        js, de = oracle.stencil_position(np.full(r.shape, float(shift)), r)
        got = oracle.interpolate(x, js, de, 8)
        np.testing.assert_allclose(got, x[r - shift], rtol=0, atol=1e-14)


def test_interpolation_equals_printed_alternating_form():
    """The oracle's sinc form against the paper's printed form
    sin(pi delta_j0)/pi sum (-1)^(j-j0) x_j w_j / delta_j, j0 = j* - D."""
    rng = np.random.default_rng(4)
    D = 8
    x = rng.standard_normal(300) + 1j * rng.standard_normal(300)
    n = np.arange(2 * D + 1)
    w = 0.54 - 0.46 * np.cos(np.pi * n / D)
    for _ in range(200):
        r = int(rng.integers(40, 260))
        e = rng.uniform(-20, 20)
        t = r - e                          # t / dt
        jstar = int(math.floor(t + 0.5))
        j0 = jstar - D
        j = np.arange(jstar - D, jstar + D + 1)
        dj = t - j
        if np.min(np.abs(dj)) < 1e-9:
            continue
        printed = math.sin(math.pi * dj[0]) / math.pi * np.sum((-1.0) ** (j - j0) * x[j] * w / dj)
        got = oracle.interpolate(x, *oracle.stencil_position(np.array([e]), np.array([r])), D)[0]
        assert abs(got - printed) < 1e-10 * max(1.0, abs(printed))


def _tone_error(D, nus, rng, n_off=64):
    worst = 0.0
    N = 400
    j = np.arange(N)
    for nu in nus:
        x = np.exp(2j * np.pi * nu * j)
        r = np.full(n_off, 200)
        e = rng.uniform(-0.5, 0.5, n_off) + 17.0
        got = oracle.interpolate(x, *oracle.stencil_position(e, r), D)
        exact = np.exp(2j * np.pi * nu * (r - e))
        worst = max(worst, np.max(np.abs(got - exact)))
    return worst


def test_interpolation_band_limited_tone_error():
    """Windowed-sinc converges as D grows; at D = 8 the error on tones up to 0.35
    cycles/sample is about 1e-2 (the paper's typical D, Sec. III A 1) and it
    shrinks with every doubling of D."""
    rng = np.random.default_rng(5)
    nus = np.linspace(0.0, 0.35, 15)
    e8 = _tone_error(8, nus, rng)
    e16 = _tone_error(16, nus, rng)
    e32 = _tone_error(32, nus, rng)
    assert e8 < 1.5e-2
    assert e16 < 5e-3
    assert e32 < e16 < e8


# ---------------------------------------------------------------------------
# Timing (Eqs. t-ssb-equation, tau-equation)
# ---------------------------------------------------------------------------
def _real_det(n=20000):
    cfg = SearchConfig(t0=synth.T0_GPS, dt=1.0, n_samples=n, f_h=100.0, f_band=1.0,
                       T_sft=240.0, T_max=0.0)
    return cfg, synth.make_detector_tables(synth.H1, cfg, np.ones(100))


def test_delay_round_trip_through_forward_model():
    cfg, det = _real_det()
    rng = np.random.default_rng(6)
    tau = rng.uniform(0, 19000, 2000)
    a_p, P = 1.44, synth.SCO_X1_P
    tasc = synth.T_ASC_O1 - cfg.t0 + 12.3
    d = oracle.delay(det, a_p, tasc, P, tau)
    t = tau - d
    # forward model written out: tau(t) = t_SSB - a_p sin(2 pi (t_SSB - T_asc)/P)
    u = (t - det.eph_t0) / det.eph_dt
    i = np.floor(u).astype(int)
    dl = det.ssb_delay[i] + (u - i) * (det.ssb_delay[i + 1] - det.ssb_delay[i])
    tssb = t + dl
    tau_back = tssb - a_p * np.sin(2 * np.pi * (tssb - tasc) / P)
    assert np.max(np.abs(tau_back - tau)) < 1e-9
    assert np.max(np.abs(d)) > 100.0          # a real Roemer delay was exercised


def test_delay_special_cases():
    cfg, det = _real_det()
    tau = np.linspace(0, 19000, 777)
    det.ssb_delay[:] = 3.25                    # constant SSB offset, no orbit
    np.testing.assert_allclose(oracle.delay(det, 0.0, 0.0, 1e5, tau), 3.25, atol=1e-15)
    det.ssb_delay[:] = 0.0                     # orbit alone: t = t_SSB, circular orbit
    a_p, P, tasc = 1.5, 68023.7, 500.0
    d = oracle.delay(det, a_p, tasc, P, tau)
    u = tau - d
    np.testing.assert_allclose(u - a_p * np.sin(2 * np.pi * (u - tasc) / P), tau, atol=1e-10)
    assert np.max(np.abs(d)) > 1.4


# ---------------------------------------------------------------------------
# Spectra, pairs, normalisation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("f_h", [120.0, 120.3])      # f_h dt' not an integer: the heterodyne matters
@pytest.mark.parametrize("f_band", [0.5, 0.05, 0.37])
def test_direct_dft_equals_fft_route(f_band, f_h):
    cfg = SearchConfig(t0=0.0, dt=1.0, n_samples=2048, f_h=f_h, f_band=f_band,
                       T_sft=64.0, T_max=128.0, T_short=128.0)
    p = oracle.make_plan(cfg)
    rng = np.random.default_rng(7)
    y = rng.standard_normal(2048) + 1j * rng.standard_normal(2048)
    a = oracle.spectra_direct(y, p)
    b = oracle.spectra_fft(y, p)
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(a))


def test_tone_on_output_bin_sums_coherently():
    """A tone exactly at an output frequency: every segment's spectrum at that bin is
    the plain sum of its samples (all phases cancel: Phi_in, f_r*, k0 bookkeeping)."""
    cfg = SearchConfig(t0=0.0, dt=1.0, n_samples=4096, f_h=120.0, f_band=0.05,
                       T_sft=64.0, T_max=128.0, T_short=128.0)
    p = oracle.make_plan(cfg)
    rng = np.random.default_rng(8)
    k = p.N_f // 3
    r = np.arange(p.M * p.N_s)
    amp = rng.uniform(0.5, 1.5, r.size)
    y = amp * np.exp(2j * np.pi * p.dfreq[k] * r)
    F = oracle.spectra_fft(y, p)
    expect = amp.reshape(p.M, p.N_s).sum(axis=1)
    np.testing.assert_allclose(F[:, k], expect, rtol=1e-10)


def test_pair_set_against_brute_enumeration():
    for Q, M, R in ((2, 7, 1), (3, 6, 2), (2, 5, 0), (1, 6, 3)):
        items = [(X, K) for X in range(Q) for K in range(M)]
        un = {(a, b) for a, b in itertools.combinations(items, 2) if abs(a[1] - b[1]) <= R}
        got = {((X, K), (Y, L)) for X, K, Y, L in oracle.pair_list(Q, M, R, oracle.PAIR_UNORDERED)}
        got_sym = {tuple(sorted(p)) for p in got}
        assert got_sym == {tuple(sorted(p)) for p in un} and len(got) == len(un)
        cross = {tuple(sorted(p)) for p in un if p[0][0] != p[1][0]}
        got_c = {tuple(sorted(((X, K), (Y, L))))
                 for X, K, Y, L in oracle.pair_list(Q, M, R, oracle.PAIR_CROSS_ONLY)}
        assert got_c == cross
        allp = {(a, b) for a in items for b in items if abs(a[1] - b[1]) <= R}
        got_a = {((X, K), (Y, L)) for X, K, Y, L in oracle.pair_list(Q, M, R, oracle.PAIR_ALL_ORDERED)}
        assert got_a == allp


def test_fstat_factorisation_and_unordered_identity():
    """All ordered pairs incl. auto-correlation over the whole span give
    |sum F_a|^2 + |sum F_b|^2 (Appendix A, F-statistic limit); the default
    unordered set is half of that minus the auto terms."""
    rng = np.random.default_rng(9)
    Q, M, nf = 2, 5, 11
    cfg = SearchConfig(t0=0.0, dt=1.0, n_samples=M * 16, f_h=100.0, f_band=0.01,
                       T_sft=16.0, T_max=16.0 * M, T_short=16.0)
    p = oracle.make_plan(cfg)
    p.N_f = nf
    Fa = [rng.standard_normal((M, nf)) + 1j * rng.standard_normal((M, nf)) for _ in range(Q)]
    Fb = [rng.standard_normal((M, nf)) + 1j * rng.standard_normal((M, nf)) for _ in range(Q)]
    Sa = sum(f.sum(axis=0) for f in Fa)
    Sb = sum(f.sum(axis=0) for f in Fb)
    auto = sum((np.abs(f) ** 2).sum(axis=0) for f in Fa + Fb)
    allp = oracle.pair_sum(Fa, Fb, p, oracle.PAIR_ALL_ORDERED)
    np.testing.assert_allclose(allp, np.abs(Sa) ** 2 + np.abs(Sb) ** 2, rtol=1e-12)
    un = oracle.pair_sum(Fa, Fb, p, oracle.PAIR_UNORDERED)
    np.testing.assert_allclose(un, 0.5 * (np.abs(Sa) ** 2 + np.abs(Sb) ** 2 - auto), rtol=1e-11)


def test_recovered_power_matches_paper():
    """Zero-padding to T_FFT and one bin per frequency recover <Xi^2> = 0.861, 0.963
    and 0.983 of rho for T_FFT = 1, 2, 3 T_coh with T_coh = 3 T_short, averaged over
    a uniform offset from the bin (Sec. III B 3)."""
    g = _golden("paper_printed_values.json")["recovered_power_resamp"]
    Ns, M = 64, 64
    cfg = SearchConfig(t0=0.0, dt=1.0, n_samples=Ns * M, f_h=100.0, f_band=0.2,
                       T_sft=Ns, T_max=Ns, T_short=Ns, pair_mode=oracle.PAIR_CROSS_ONLY)
    # the paper's set-up: pairs up to T_max = T_short span T_coh = 3 T_short
    assert oracle.make_plan(cfg).T_coh == g["T_coh_over_T_short"] * Ns
    kappas = (np.arange(48) + 0.5) / 48 - 0.5
    for mult, expect in zip((1, 2, 3), g["values"]):
        p = oracle.make_plan(cfg, n_fft=3 * Ns * mult)
        k = p.N_f // 2
        r = np.arange(p.M * p.N_s)
        vals = []
        for kap in list(kappas) + [0.0]:
            x = np.exp(2j * np.pi * (p.dfreq[k] + kap / p.T_FFT) * r)
            ds = _flat_dataset(cfg, np.stack([x, x]))
            vals.append(oracle.rho_template(ds, ds.templates[0], p)[k])
        ratio = np.mean(vals[:-1]) / vals[-1]
        assert abs(ratio - expect) < g["tolerance"], (mult, ratio, expect)


# ---------------------------------------------------------------------------
# Whole statistic
# ---------------------------------------------------------------------------
def _zero_roemer_tiny(seed, noise, inj=None, n=4096, sigma_jitter=0.2, duty=0.85):
    ds = synth.tiny(seed=seed, n_samples=n, noise=noise, injection=inj, zero_roemer=True,
                    const_ab=(0.7, -0.4), sigma_jitter=sigma_jitter, duty=duty,
                    templates=np.array([[0.0, synth.T_ASC_O1, synth.SCO_X1_P]]))
    return ds


def test_noise_block_against_exact_floor():
    """The T_sft block of detector time t = (j* + delta) dt' is floor((j* + delta) / nsft),
    here in exact rational arithmetic, for offsets of both signs at and near block
    boundaries (the oracle decides it from the integer j* and the sign of delta)."""
    from fractions import Fraction
    nsft = 360
    js = np.arange(-2 * nsft - 3, 2 * nsft + 4)
    for d in (-0.5, -0.3, -1e-9, 0.0, 1e-9, 0.25, 0.4999):
        got = oracle.noise_block(js, np.full(js.shape, d), nsft)
        ref = [math.floor((Fraction(int(j)) + Fraction(d)) / nsft) for j in js]
        assert list(got) == ref, d


def test_unit_variance_in_noise():
    """rho has zero mean and unit variance in Gaussian noise: the defining role of
    the normalisation N (Sec. II B)."""
    vals = []
    for s in range(40):
        ds = _zero_roemer_tiny(100 + s, noise=True)
        vals.append(oracle.rho(ds)[0])
    v = np.concatenate(vals)
    assert abs(v.mean()) < 0.06
    assert abs(v.var() - 1.0) < 0.08


def _closed_form_rho(ds, plan, k, h0, cosi, psi, phi0, a, b):
    """sqrt(2) sum_P Re(conj(s_K) s_L) / sqrt(D) for a noiseless tone on bin k with
    constant antenna functions: s_XK = e^{i phi0} h0/2 (F+ A+ - i Fx Ax) a sum alpha."""
    Fp = a * math.cos(2 * psi) + b * math.sin(2 * psi)
    Fx = b * math.cos(2 * psi) - a * math.sin(2 * psi)
    amp = 0.5 * h0 * (Fp * 0.5 * (1 + cosi ** 2) - 1j * Fx * cosi) * np.exp(1j * phi0)
    nsft = int(round(ds.cfg.T_sft))
    sa, sb, nA, nB, nC = [], [], [], [], []
    for det in ds.dets:
        sig = np.repeat(det.sigma, nsft)[: plan.M * plan.N_s]
        w = np.where(sig > 0, 1.0 / np.where(sig > 0, sig, 1.0) ** 2, 0.0)
        s2 = sig ** 2
        seg = lambda v: v.reshape(plan.M, plan.N_s).sum(axis=1)
        sa.append(amp * a * seg(w))
        sb.append(amp * b * seg(w))
        nA.append(seg(a * a * w * w * s2))
        nB.append(seg(b * b * w * w * s2))
        nC.append(seg(a * b * w * w * s2))
    num, den = 0.0, 0.0
    Q = len(ds.dets)
    for X in range(Q):
        for Y in range(Q):
            for K in range(plan.M):
                for L in range(plan.M):
                    ok = (X < Y and abs(K - L) <= plan.R) or (X == Y and 1 <= L - K <= plan.R)
                    if ok:
                        num += (np.conj(sa[X][K]) * sa[Y][L] + np.conj(sb[X][K]) * sb[Y][L]).real
                        den += nA[X][K] * nA[Y][L] + nB[X][K] * nB[Y][L] + 2 * nC[X][K] * nC[Y][L]
    return math.sqrt(2.0) * num / math.sqrt(den)


def test_noiseless_injection_closed_form_zero_roemer():
    base = _zero_roemer_tiny(1, noise=False)
    p = oracle.make_plan(base.cfg)
    k = 123
    inj = Injection(h0=0.3, f0=p.freq[k], a_p=0.0, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P,
                    cosi=0.4, psi=0.9, phi0=1.1)
    ds = _zero_roemer_tiny(1, noise=False, inj=inj)
    got = oracle.rho(ds)[0]
    expect = _closed_form_rho(ds, p, k, 0.3, 0.4, 0.9, 1.1, 0.7, -0.4)
    assert abs(got[k] - expect) < 1e-9 * abs(expect)
    assert int(np.argmax(got)) == k


def test_noiseless_closed_form_time_varying_antenna_functions():
    """Zero Roemer delay, real a(t), b(t) tabulated at every sample (ab_dt = dt) and
    gaps: the spectra at the injected bin are sums of weighted amplitudes with
    alpha_r = a(t_r)/sigma^2, beta_r = b(t_r)/sigma^2 and the signal's own
    F+(t_r), Fx(t_r) -- no interpolation, no DFT phase survives."""
    kw = dict(seed=4, noise=False, zero_roemer=True, ab_dt=1.0, n_samples=2 * 86400 // 16,
              T_sft=64.0, T_max=2048.0, T_short=1024.0,
              templates=np.array([[0.0, synth.T_ASC_O1, synth.SCO_X1_P]]))
    p = oracle.make_plan(synth.tiny(**kw).cfg)
    k = 57
    inj = Injection(h0=0.4, f0=p.freq[k], a_p=0.0, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P,
                    cosi=-0.3, psi=0.2, phi0=2.0)
    ds = synth.tiny(injection=inj, **kw)
    p = oracle.make_plan(ds.cfg)
    got = oracle.rho(ds)[0]
    nsft = 64
    A_p, A_x = 0.5 * (1 + inj.cosi ** 2), inj.cosi
    c2, s2p = math.cos(2 * inj.psi), math.sin(2 * inj.psi)
    n = p.M * p.N_s
    sa, sb, nA, nB, nC = [], [], [], [], []
    seg = lambda v: v.reshape(p.M, p.N_s).sum(axis=1)
    for det in ds.dets:
        a, b = det.a_tab[:n], det.b_tab[:n]
        sig = np.repeat(det.sigma, nsft)[:n]
        w = np.where(sig > 0, 1.0 / np.where(sig > 0, sig, 1.0) ** 2, 0.0)
        h = 0.5 * inj.h0 * ((a * c2 + b * s2p) * A_p - 1j * (b * c2 - a * s2p) * A_x)
        h = h * np.exp(1j * inj.phi0) * (sig > 0)
        sa.append(seg(a * w * h))
        sb.append(seg(b * w * h))
        nA.append(seg(a * a * w * w * sig ** 2))
        nB.append(seg(b * b * w * w * sig ** 2))
        nC.append(seg(a * b * w * w * sig ** 2))
    num = den = 0.0
    for X, K, Y, L in itertools.product(range(2), range(p.M), range(2), range(p.M)):
        if (X < Y and abs(K - L) <= p.R) or (X == Y and 1 <= L - K <= p.R):
            num += (np.conj(sa[X][K]) * sa[Y][L] + np.conj(sb[X][K]) * sb[Y][L]).real
            den += nA[X][K] * nA[Y][L] + nB[X][K] * nB[Y][L] + 2 * nC[X][K] * nC[Y][L]
    expect = math.sqrt(2.0) * num / math.sqrt(den)
    assert abs(got[k] - expect) < 1e-9 * abs(expect)


def test_noiseless_injection_realistic_timing_and_scaling():
    """With real Roemer delays the on-template rho recovers the zero-Roemer closed
    form within the D = 8 interpolation deficit; the argmax is the injected
    (template, bin); rho scales as h0^2 (Appendix C)."""
    probe = synth.tiny(seed=2, noise=False)
    p = oracle.make_plan(probe.cfg)
    k = 201
    tasc = synth.T_ASC_O1 + 17.0
    inj = Injection(h0=0.3, f0=p.freq[k], a_p=1.44, T_asc=tasc, P=synth.SCO_X1_P,
                    cosi=0.4, psi=0.9, phi0=1.1)
    tm = np.array([[1.44, tasc, synth.SCO_X1_P], [1.30, tasc, synth.SCO_X1_P],
                   [1.44, tasc + 900.0, synth.SCO_X1_P]])
    kw = dict(seed=2, noise=False, const_ab=(0.7, -0.4), templates=tm)
    ds = synth.tiny(injection=inj, **kw)
    got = oracle.rho(ds)
    # the same tone with neither Earth nor orbital Roemer delay: resampling is exact
    ref = synth.tiny(injection=Injection(**{**inj.__dict__, "a_p": 0.0}), zero_roemer=True, **kw)
    ref.templates = np.array([[0.0, tasc, synth.SCO_X1_P]])
    expect = oracle.rho(ref)[0][k]
    assert abs(got[0, k] / expect - 1.0) < 0.02
    ti, bi = np.unravel_index(np.argmax(got), got.shape)
    assert (ti, bi) == (0, k)
    inj2 = Injection(**{**inj.__dict__, "h0": 0.6})
    got2 = oracle.rho(synth.tiny(injection=inj2, **kw))
    np.testing.assert_allclose(got2, 4.0 * got, rtol=1e-9, atol=1e-9 * np.abs(got).max())


def test_invariances():
    """Orbital period shift of T_asc, detector swap, and a whole-segment shift of the
    time origin leave rho unchanged (the statistic depends on relative time only)."""
    ds = synth.tiny(seed=5, noise=True, n_templates=2,
                    injection=Injection(h0=0.2, f0=120.07, a_p=1.44, T_asc=synth.T_ASC_O1,
                                        P=synth.SCO_X1_P))
    base = oracle.rho(ds)
    tm = ds.templates.copy()
    tm[:, 1] += tm[:, 2]
    np.testing.assert_allclose(oracle.rho(ds, templates=tm), base, atol=1e-8)
    sw = Dataset(ds.cfg, ds.dets[::-1], ds.x[::-1].copy(), ds.templates)
    np.testing.assert_allclose(oracle.rho(sw), base, atol=1e-10)
    # shift the origin one segment earlier (prepend N_s empty samples); the first and
    # last 768 s are gaps, wider than the Roemer delay, so both grids see the same data
    p = oracle.make_plan(ds.cfg)
    ns = p.N_s
    nsft = int(round(ds.cfg.T_sft))
    edge = 768 // nsft
    for q, d in enumerate(ds.dets):
        d.sigma[:edge] = 0.0
        d.sigma[-edge:] = 0.0
        ds.x[q, :edge * nsft] = 0.0
        ds.x[q, -edge * nsft:] = 0.0
    base = oracle.rho(ds)
    cfg2 = SearchConfig(**{**ds.cfg.__dict__, "t0": ds.cfg.t0 - ns, "n_samples": ds.cfg.n_samples + ns})
    dets2 = []
    for d in ds.dets:
        d2 = synth.DetectorTables(d.name, d.eph_t0 + ns, d.eph_dt, d.ssb_delay, d.ab_t0 + ns,
                                  d.ab_dt, d.a_tab, d.b_tab,
                                  np.concatenate([np.zeros(ns // nsft), d.sigma]))
        dets2.append(d2)
    x2 = np.concatenate([np.zeros((2, ns), complex), ds.x], axis=1)
    sh = Dataset(cfg2, dets2, x2, ds.templates)
    np.testing.assert_allclose(oracle.rho(sh), base, atol=1e-8)


def test_detector_frame_brute_force():
    """The resampled rho against the detector-frame sum over raw samples (no
    interpolation): zero Roemer gives equality to rounding; real delays agree to
    the resampling accuracy with the same argmax (Sec. III B 6)."""
    probe = synth.tiny(seed=3, noise=False, n_samples=8192, T_sft=256.0, T_max=512.0,
                       T_short=512.0, D=16)
    p = oracle.make_plan(probe.cfg)
    k = 77
    tasc = synth.T_ASC_O1 - 33.0
    inj = Injection(h0=0.5, f0=p.freq[k], a_p=1.44, T_asc=tasc, P=synth.SCO_X1_P,
                    cosi=0.2, psi=0.4, phi0=0.3)
    tm = np.array([[1.44, tasc, synth.SCO_X1_P]])
    kw = dict(seed=3, n_samples=8192, T_sft=256.0, T_max=512.0, T_short=512.0, D=16,
              templates=tm, duty=1.0, sigma_jitter=0.0)
    zr = synth.tiny(noise=True, zero_roemer=True, const_ab=(0.5, 0.3), **kw)
    zr.templates = np.array([[0.0, tasc, synth.SCO_X1_P]])
    np.testing.assert_allclose(oracle.detector_frame_rho(zr, zr.templates[0]),
                               oracle.rho_template(zr, zr.templates[0]), atol=1e-9)
    ds = synth.tiny(noise=False, injection=inj, **kw)
    res = oracle.rho_template(ds, tm[0])
    det = oracle.detector_frame_rho(ds, tm[0])
    scale = np.max(np.abs(res))
    assert np.max(np.abs(res - det)) < 5e-3 * scale
    assert int(np.argmax(res)) == int(np.argmax(det)) == k


def test_topk_order_and_ties():
    rho = np.array([[1.0, 3.0, 2.0], [3.0, 0.5, 2.0]])
    t, b, v = oracle.topk(rho, 4)
    assert list(zip(t, b)) == [(0, 1), (1, 0), (0, 2), (1, 2)]
    assert list(v) == [3.0, 3.0, 2.0, 2.0]
