"""Pins of the oracle's learned 8-tap interpolator (oracle.learned).

The paper has no learned interpolator, so nothing it prints pins this one: its parity
against the paper is unpinned.  What pins the oracle's evaluation of the network is
interpolation itself: a trained network must reproduce band-limited tones to within
its training error, and a transposed layer, a wrong activation, a wrong tap offset or a
wrong input scaling each turn that into an O(1) error.  Its rho is then judged against
the exact D = 16 windowed sinc."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from oracle import learned
from paper_1712_06515_gb300 import learned_interp

MODEL = learned.load(learned_interp.WEIGHTS)
NU_C = 0.2875          # 0.5 Hz band at 150 Hz, 1 s sampling


def _tone_errors(nu_c, n=20000, seed=5):
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, n)
    nu = rng.uniform(-nu_c, nu_c, n)
    j = np.arange(8) - 3
    est = (learned.taps(MODEL, u, nu_c) * np.exp(2j * np.pi * nu[:, None] * j)).sum(1)
    return np.abs(est - np.exp(2j * np.pi * nu * u))


@pytest.mark.parametrize("nu_c", [0.16, 0.2, NU_C, 0.31])
def test_taps_reproduce_band_limited_tones(nu_c):
    e = _tone_errors(nu_c)
    # the stored network's accuracy (max 8.3e-3, rms 1.5e-3 at nu_c = 0.31; 4.1e-3 and
    # 8.4e-4 at 0.2875) with margin; the exact D = 8 stencil: max 1.2e-2, rms 4.5e-3 at 0.2875
    assert e.max() < 1.2e-2
    assert np.sqrt(np.mean(e ** 2)) < 2.5e-3


def test_taps_near_interpolating_at_integer_offset():
    # at u = 0 the point is sample floor(t) itself: tap 3 near one, the others near zero
    c = learned.taps(MODEL, np.array([0.0]), NU_C)[0]
    assert abs(c[3] - 1.0) < 2e-2
    assert np.all(np.abs(np.delete(c, 3)) < 2e-2)


def test_interpolate_positions_both_signs_of_delta():
    # a tone series sampled at integers, evaluated at t = j* + delta for delta on both
    # sides of zero: checks floor(t) and u as the interpolator derives them from (j*, delta)
    rng = np.random.default_rng(11)
    N = 256
    nu = 0.17
    x = np.exp(2j * np.pi * nu * np.arange(N))
    jstar = rng.integers(8, N - 8, 4000)
    delta = rng.uniform(-0.5, 0.5, 4000)
    est = learned.interpolate(x, jstar, delta, MODEL, NU_C)
    exact = np.exp(2j * np.pi * nu * (jstar + delta))
    assert np.max(np.abs(est - exact)) < 1e-2
    # the edge: samples outside [0, N) are zero, so near t = 0 only the in-range taps count
    e0 = learned.interpolate(x, np.array([0]), np.array([0.25]), MODEL, NU_C)[0]
    c = learned.taps(MODEL, np.array([0.25]), NU_C)[0]
    assert abs(e0 - np.sum(c[3:] * x[:5])) < 1e-12


def test_fp64_evaluation_matches_training_forward():
    # a second, independent evaluation: the training tool's PyTorch network on the same weights
    torch = pytest.importorskip("torch")
    W = [torch.tensor(w, dtype=torch.float64) for w in learned_interp.load_weights()]
    u = np.linspace(0.0, 1.0, 101)
    f = torch.tensor(learned_interp.features(u, np.full_like(u, NU_C)), dtype=torch.float64)
    h = torch.tanh(f @ W[0] + W[1])
    h = torch.tanh(h @ W[2] + W[3])
    ref = (h @ W[4] + W[5]).numpy()
    np.testing.assert_allclose(learned.taps(MODEL, u, NU_C), ref, rtol=0, atol=1e-12)


def test_learned_rho_judged_by_exact_d16_stencil():
    # noiseless injection at a realistic orbit: learned rho within 1e-2 max|rho| of the
    # D = 16 windowed sinc, at the same argmax (template, bin)
    inj = synth.Injection(h0=0.4, f0=120.1, a_p=1.44, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P)
    ds = synth.tiny(seed=41, n_templates=2, injection=inj, noise=False)
    nu_c = learned_interp.band_halfwidth(ds.cfg.f_band, ds.cfg.f_h, ds.cfg.dt)
    r16 = oracle.rho(dataclasses.replace(ds, cfg=dataclasses.replace(ds.cfg, D=16)))
    rl = oracle.rho(ds, interp=lambda x, js, d: learned.interpolate(x, js, d, MODEL, nu_c))
    assert np.abs(rl - r16).max() <= 1e-2 * max(1.0, np.abs(r16).max())
    assert np.unravel_index(rl.argmax(), rl.shape) == np.unravel_index(r16.argmax(), r16.shape)
