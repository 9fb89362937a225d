"""Pins of the oracle's elliptical-orbit timing (Eqs. solve-for-E, Kepler-equation), each
against something other than the oracle's own formulas: a bracketing root finder for
Kepler's equation, the circular limit, the first-order expansion in e, the ascending
node, the forward model's round trip, a numerical derivative, and the recovery of an
eccentric injection."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import demod

scipy_opt = pytest.importorskip("scipy.optimize")


def test_kepler_against_bracketing_root_finder():
    rng = np.random.default_rng(3)
    for e in (1e-3, 0.1, 0.5, 0.9):
        M = rng.uniform(-10.0, 10.0, 40)
        E = oracle.kepler_E(M, e)
        for m, ee in zip(M, E):
            ref = scipy_opt.brentq(lambda x: x - e * math.sin(x) - m, m - 1.0, m + 1.0, xtol=1e-15, rtol=1e-15)
            assert abs(ee - ref) < 1e-12


def test_circular_limit_for_any_omega():
    u = np.linspace(-3e5, 3e5, 777)
    circ = 1.44 * np.sin(2 * np.pi * (u - 1234.5) / 68023.7)
    for w in (0.0, 0.7, -2.9):
        # e -> 0 with the periapsis placed from T_asc: the same circular orbit
        got = oracle.binary_delay(1.44, 1234.5, 68023.7, u, 1e-14, w)
        np.testing.assert_allclose(got, circ, rtol=0, atol=1e-12)


def test_first_order_expansion_in_e():
    a_p, P, w, e = 1.7, 50000.0, 0.9, 1e-4
    tasc = 321.0
    Tp = oracle.periapsis_time(tasc, P, e, w)
    u = np.linspace(0.0, 2 * P, 1001)
    M = 2 * np.pi * (u - Tp) / P
    approx = a_p * (np.sin(M + w) + 0.5 * e * np.sin(2 * M + w) - 1.5 * e * math.sin(w))
    got = oracle.binary_delay(a_p, tasc, P, u, e, w)
    assert np.abs(got - approx).max() < 3 * a_p * e * e


@pytest.mark.parametrize("e,w", [(0.05, 0.3), (0.4, 2.0), (0.7, -1.2)])
def test_ascending_node_at_T_asc(e, w):
    a_p, P, tasc = 1.44, 68023.7, 5000.0
    assert abs(oracle.binary_delay(a_p, tasc, P, np.array([tasc]), e, w)[0]) < 1e-12
    h = 1.0
    up = oracle.binary_delay(a_p, tasc, P, np.array([tasc - h, tasc + h]), e, w)
    assert up[1] > up[0]            # ascending: moving away from the observer


def test_eccentric_delay_round_trip_and_derivative():
    ds = synth.tiny(seed=5, n_templates=1)
    det = ds.dets[0]
    a_p, tasc, P, e, w = 1.44, synth.T_ASC_O1 - ds.cfg.t0, synth.SCO_X1_P, 0.35, 0.8
    tau = np.linspace(0.0, 4000.0, 301)
    d = oracle.delay(det, a_p, tasc, P, tau, e, w)
    t = tau - d
    # forward model: tau(t) = t + Delta(t) - R(t + Delta(t))/c
    fwd = t + oracle.ssb_delay(det, t) - oracle.binary_delay(a_p, tasc, P, t + oracle.ssb_delay(det, t), e, w)
    assert np.abs(fwd - tau).max() < 1e-9
    # dtau/dt of the detector-frame model against a central difference of the forward model
    tq = np.linspace(100.0, 3900.0, 50)
    dd, dtau = demod.source_time(det, a_p, tasc, P, tq, e, w)
    h = 1e-3
    f = lambda x: x + oracle.ssb_delay(det, x) - oracle.binary_delay(a_p, tasc, P, x + oracle.ssb_delay(det, x), e, w)
    np.testing.assert_allclose(dtau, (f(tq + h) - f(tq - h)) / (2 * h), rtol=0, atol=1e-9)
    np.testing.assert_allclose(tq + dd, f(tq), rtol=0, atol=1e-9)


def test_eccentric_injection_recovered_by_its_template():
    inj = synth.Injection(h0=0.5, f0=120.1, a_p=1.44, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P, e=0.3, omega=1.1)
    tm = np.array([[inj.a_p, inj.T_asc, inj.P, inj.e, inj.omega],
                   [inj.a_p, inj.T_asc, inj.P, 0.0, 0.0]])
    ds = synth.tiny(seed=7, n_samples=8192, noise=False, injection=inj, templates=tm)
    r = oracle.rho(ds)
    p = oracle.make_plan(ds.cfg)
    k = int(np.argmin(np.abs(p.freq - inj.f0)))
    assert int(r[0].argmax()) == k
    assert r[0].max() > 1.2 * r[1].max()
