"""Pins of the detector-frame ("demodulation") oracle, oracle/demod.py, each independent
of the oracle's own formulas: the SFT convention against the closed-form DFT of a tone,
the sinc data vector's phase and size against a tone of known phase at the SFT
mid-time, the pair set against its closed-form count, unit variance in noise (the role
of N), h0^2 scaling, the argmax on the injection, and the invariances."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import demod

INJ = synth.Injection(h0=0.4, f0=120.1, a_p=1.44, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P)


def test_sft_matches_closed_form_dft_of_a_tone():
    ds = synth.tiny(seed=3, n_templates=1, noise=False, duty=1.0, sigma_jitter=0.0)
    N = int(ds.cfg.T_sft / ds.cfg.dt)
    nu = 0.0377                                   # cycles per sample
    j = np.arange(ds.cfg.n_samples)
    x = np.exp(2j * np.pi * nu * j)
    ds = dataclasses.replace(ds, x=[x, x])
    ks, tmid, z, sig = demod.sfts(ds)[0]
    k = ks[3]
    m = np.fft.fftfreq(N, 1.0 / N)                # bin numbers in FFT order
    # sum_{j<N} exp(2 pi i (nu - m/N) (kN + j)) dt, summed as a geometric series
    r = np.exp(2j * np.pi * (nu - m / N))
    geo = np.exp(2j * np.pi * nu * k * N) * (1 - r ** N) / (1 - r) * ds.cfg.dt
    S = 2.0 * sig[3] ** 2 * ds.cfg.dt
    np.testing.assert_allclose(z[3], geo * math.sqrt(2.0 / (ds.cfg.T_sft * S)), rtol=0, atol=1e-9)
    assert abs(tmid[3] - (k * N + N / 2) * ds.cfg.dt) < 1e-12


@pytest.mark.parametrize("xpos", [3.3, -7.75, 0.5, 12.0])
def test_data_vector_recovers_tone_phase_and_size(xpos):
    """A tone with heterodyned frequency x / T_sft and phase phi at the SFT mid-time gives
    z_K = A T sqrt(2/(T S)) Xi_K exp(i phi) up to the Dirichlet-vs-sinc difference."""
    T, dt = 360.0, 1.0
    N = int(T / dt)
    phi = 0.9
    t = dt * np.arange(N) - T / 2                 # relative to the mid-time
    x = 1.7 * np.exp(1j * (phi + 2 * np.pi * (xpos / T) * t))
    S = 2.0 * 1.0 * dt
    z = (np.fft.fft(x) * dt * math.sqrt(2.0 / (T * S)))[None, :]
    zK, xi = demod.sft_data_vector(z, np.array([[xpos]]), n_bin=2)
    expect = 1.7 * T * math.sqrt(2.0 / (T * S)) * xi[0, 0]
    assert abs(np.angle(zK[0, 0] * np.exp(-1j * phi))) < 5e-3
    assert abs(abs(zK[0, 0]) / expect - 1.0) < 5e-3


def test_pair_set_count_closed_form():
    ds = synth.tiny(seed=3, n_templates=1, duty=1.0)
    n = min(len(ds.dets[0].sigma), ds.cfg.n_samples // int(ds.cfg.T_sft))
    Rs = int(ds.cfg.T_max // ds.cfg.T_sft)
    lagged = n * Rs - Rs * (Rs + 1) // 2          # pairs (k, l), 0 < l - k <= Rs, per detector pair
    expect = 2 * lagged + (n + 2 * lagged)        # two same-detector sets, then cross: same time + both lags
    pairs = demod.pair_list(ds)
    assert len(pairs) == expect
    assert len(set(pairs)) == len(pairs)
    assert all((X, k) != (Y, l) for X, k, Y, l in pairs)


def test_unit_variance_in_noise():
    vals = []
    for seed in range(6):
        ds = synth.tiny(seed=100 + seed, n_templates=4)
        for tm in ds.templates:
            r = demod.demod_rho(ds, tm)
            vals.append(r[::7])                   # bins 7 apart: nearly independent
    v = np.concatenate(vals)
    assert abs(v.mean()) < 4.0 / math.sqrt(len(v)) * 1.5
    assert abs(v.var() - 1.0) < 0.12


def test_injection_argmax_and_h0_squared_scaling():
    ds = synth.tiny(seed=41, n_templates=3, injection=INJ, noise=False)
    r = np.stack([demod.demod_rho(ds, tm) for tm in ds.templates])
    ti, bi = np.unravel_index(r.argmax(), r.shape)
    ref = oracle.rho(ds)
    assert (ti, bi) == np.unravel_index(ref.argmax(), ref.shape)
    assert r.max() > 10.0
    ds2 = synth.tiny(seed=41, n_templates=3, injection=dataclasses.replace(INJ, h0=0.8), noise=False)
    r2 = np.stack([demod.demod_rho(ds2, tm) for tm in ds2.templates])
    np.testing.assert_allclose(r2, 4.0 * r, rtol=1e-9, atol=1e-9)


def test_invariances():
    ds = synth.tiny(seed=41, n_templates=2, injection=INJ)
    tm = ds.templates[0]
    r = demod.demod_rho(ds, tm)
    shifted = np.array([tm[0], tm[1] + tm[2], tm[2]])
    np.testing.assert_allclose(demod.demod_rho(ds, shifted), r, rtol=0, atol=1e-7)
    swapped = dataclasses.replace(ds, dets=ds.dets[::-1], x=ds.x[::-1])
    np.testing.assert_allclose(demod.demod_rho(swapped, tm), r, rtol=0, atol=1e-9)


def test_signal_bins_follow_the_doppler_shifted_tone():
    """Each SFT's power peak of a noiseless injection (the maximum of its 64-times
    zero-padded transform) sits at the bin position the signal model predicts."""
    inj = synth.Injection(h0=1.0, f0=150.05, a_p=1.44, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P)
    ds = synth.tiny(seed=9, n_samples=360 * 24, T_sft=360.0, T_max=720.0, T_short=720.0, f_h=150.0,
                    duty=1.0, noise=False, injection=inj, n_templates=1)
    ks, tmid, z, _ = demod.sfts(ds)[0]
    x, _ = demod.signal_bins(ds.dets[0], ds.cfg, inj.a_p, inj.T_asc - ds.cfg.t0, inj.P, tmid, np.array([inj.f0]))
    N, pad = z.shape[1], 64
    shifts = []
    for i, k in enumerate(ks):
        seg = ds.x[0][k * N:(k + 1) * N]
        spec = np.abs(np.fft.fft(seg, N * pad)) ** 2
        j = int(np.argmax(spec))
        peak = (j if j < N * pad // 2 else j - N * pad) / pad
        assert abs(peak - x[i, 0]) < 0.05, (i, peak, x[i, 0])
        shifts.append(peak - (inj.f0 - ds.cfg.f_h) * ds.cfg.T_sft)
    assert np.ptp(shifts) > 1.0          # the Doppler shift moves the tone by bins over the day


def test_equals_resampled_statistic_where_the_two_coincide():
    """No Roemer delay, no orbit, T_max = 0 and T_short = T_sft: both statistics
    cross-correlate the same-time blocks of the two detectors; for a tone on an SFT bin
    the sinc kernel is exact and the antenna weights are those of the resampled a, b at
    the mid-time, so the two rho agree at the tone's frequency to the change of a, b
    within one block."""
    dt, T = 1.0, 64.0
    f0 = 120.0 + 5.0 / T
    inj = synth.Injection(h0=0.5, f0=f0, a_p=0.0, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P)
    ds = synth.tiny(seed=12, T_sft=T, T_max=0.0, T_short=T, zero_roemer=True, noise=False, duty=1.0,
                    injection=inj, templates=np.array([[0.0, synth.T_ASC_O1, synth.SCO_X1_P]]))
    rd = demod.demod_rho(ds, ds.templates[0], freqs=np.array([f0]))
    p = oracle.make_plan(ds.cfg)
    import oracle.crosscorr as oc
    # the resampled statistic at the same frequency, from the oracle's direct DFT
    plan_f = dataclasses.replace(p, freq=np.array([f0]), dfreq=np.array([f0 - ds.cfg.f_h]), N_f=1)
    rr = oc.rho_template(ds, ds.templates[0], plan=plan_f, spectra="direct")
    assert rd[0] > 10.0
    assert abs(rd[0] / rr[0] - 1.0) < 2e-3, (rd[0], rr[0])


@pytest.mark.parametrize("kw", [dict(), dict(T_max=256.0, T_short=128.0), dict(n_det=3, duty=0.6)])
def test_separable_rearrangement_equals_pair_loop(kw):
    """The separable form the GPU offers beside the pair loop: with
    Gamma_KL = (a^_K a^_L + b^_K b^_L) / 10, the pair sum of SFT K over its partners L is
    2 Re(conj(y_K) (a^_K S_A + b^_K S_B)) / 10 (S_A = sum_L a^_L y_L, S_B likewise) and its
    normalisation term Xi_K^2 (a^_K^2 U_AA + 2 a^_K b^_K U_AB + b^_K^2 U_BB) / 100
    (U_AA = sum_L Xi_L^2 a^_L^2, ...).  Built here from the oracle's own pieces and summed
    over the partner windows directly, it equals the oracle's pair loop to FP64 rounding."""
    ds = synth.tiny(seed=19, n_templates=2, injection=INJ, **kw)
    cfg = ds.cfg
    plan = oracle.make_plan(cfg)
    f = plan.freq
    for tmpl in ds.templates:
        a_p, tasc, P, e, omega = oracle.orbit(tmpl)
        T, Y, XI, AH, BH = [], [], [], [], []
        for det, (ks, tmid, z, sig) in zip(ds.dets, demod.sfts(ds)):
            if len(ks) == 0:
                continue
            x, cyc = demod.signal_bins(det, cfg, a_p, tasc - cfg.t0, P, tmid, f, e, omega)
            zK, xi = demod.sft_data_vector(z, x)
            Y.append(xi * zK * np.exp(-2j * np.pi * cyc))
            XI.append(xi)
            scale = np.sqrt(2.0 * cfg.T_sft / (2.0 * sig * sig * cfg.dt))
            AH.append(scale * demod._lerp(det.ab_t0, det.ab_dt, det.a_tab, tmid))
            BH.append(scale * demod._lerp(det.ab_t0, det.ab_dt, det.b_tab, tmid))
            T.append(tmid)
        T = np.concatenate(T)
        order = np.argsort(T, kind="stable")
        T, Y, XI = T[order], np.concatenate(Y)[order], np.concatenate(XI)[order]
        AH, BH = np.concatenate(AH)[order], np.concatenate(BH)[order]
        raw = np.zeros(len(f))
        den = np.zeros(len(f))
        for K in range(len(T)):
            part = (np.arange(len(T)) < K) & (T[K] - T <= cfg.T_max + 1e-9)   # earlier SFTs in the window
            SA = (AH[part, None] * Y[part]).sum(axis=0)
            SB = (BH[part, None] * Y[part]).sum(axis=0)
            x2 = XI[part] ** 2
            UAA = (x2 * AH[part, None] ** 2).sum(axis=0)
            UAB = (x2 * (AH[part] * BH[part])[:, None]).sum(axis=0)
            UBB = (x2 * BH[part, None] ** 2).sum(axis=0)
            raw += 0.2 * np.real(np.conj(Y[K]) * (AH[K] * SA + BH[K] * SB))
            den += XI[K] ** 2 * (AH[K] ** 2 * UAA + 2.0 * AH[K] * BH[K] * UAB + BH[K] ** 2 * UBB) / 100.0
        sep = np.where(den > 0, raw / np.sqrt(2.0 * den), 0.0)
        ref = demod.demod_rho(ds, tmpl)
        np.testing.assert_allclose(sep, ref, rtol=0, atol=1e-9 * max(1.0, np.abs(ref).max()))
