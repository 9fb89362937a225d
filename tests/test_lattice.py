"""The parameter-space metric and template lattice (Eqs. phase-derivs-metric,
metric-spacing-eq): the oracle pinned by the many-orbit closed form and by the loss it
predicts; the library's host implementation against the oracle (no GPU needed)."""
import math

import numpy as np
import pytest

import synth
from oracle import lattice as olat

F, A_P, P = 150.0, 1.44, synth.SCO_X1_P


def lag_average(T_obs, T_sft, T_max, Q, fn):
    n = int(T_obs // T_sft)
    Rs = int(math.floor(T_max / T_sft + 1e-9))
    num = den = 0.0
    for lag in range(Rs + 1):
        mult = Q * (Q - 1) / 2 if lag == 0 else Q * Q
        num += mult * (n - lag) * fn(lag * T_sft)
        den += mult * (n - lag)
    return num / den


def test_metric_many_orbit_closed_form():
    """Averaged over many orbits (T_obs = 120 d, 152 orbits), the orbital phase is uniform:
    <(sin A - sin B)^2> = <(cos A - cos B)^2> = 1 - cos(Omega lag), cross terms vanish."""
    T_obs, T_sft, T_max, Q = 120 * 86400.0, 360.0, 3600.0, 2
    g = olat.metric(T_obs, T_sft, T_max, Q, F, A_P, 1234.0, P)
    Om = 2 * math.pi / P
    avg = lag_average(T_obs, T_sft, T_max, Q, lambda lag: 1.0 - math.cos(Om * lag))
    assert abs(g[0, 0] / (0.5 * (2 * math.pi * F) ** 2 * avg) - 1.0) < 0.01
    assert abs(g[1, 1] / (0.5 * (2 * math.pi * F * A_P * Om) ** 2 * avg) - 1.0) < 0.01
    assert abs(g[0, 1]) < 0.02 * math.sqrt(g[0, 0] * g[1, 1])
    np.testing.assert_allclose(g, g.T, rtol=1e-12)
    assert np.all(np.linalg.eigvalsh(g) > -1e-9 * np.abs(g).max())


def test_lattice_spacing_and_cover():
    g = np.diag([4.0, 0.25, 9.0])
    lo, hi = np.array([1.0, 10.0, 5.0]), np.array([2.0, 13.0, 5.0])
    L = olat.lattice(g, 0.1, lo, hi)
    d = np.sqrt(0.1 / np.diag(g))
    for i in range(3):
        ax = np.unique(L[:, i])
        assert ax[0] == lo[i] and ax[-1] >= hi[i] - 1e-12
        if len(ax) > 1:
            np.testing.assert_allclose(np.diff(ax), d[i], rtol=1e-12)
    assert len(L) == len(np.unique(L[:, 0])) * len(np.unique(L[:, 1])) * len(np.unique(L[:, 2]))


@pytest.mark.parametrize("i", [0, 1, 2])
def test_metric_predicts_the_phase_loss_of_an_offset_template(i):
    """One lattice step sqrt(mu / g_ii) away from a signal, the pairs' phase coherence
    <1 - cos(dPhi_K - dPhi_L)> drops by mu (quadratic regime): the residual phases dPhi
    taken from the injection model's orbital Roemer delay (an independent implementation)
    at the SFT mid-times, the average over the pair set of the metric."""
    T_obs, T_sft, T_max, Q = 3 * 86400.0, 360.0, 3600.0, 2
    tasc = 700.0
    g = olat.metric(T_obs, T_sft, T_max, Q, F, A_P, tasc, P)
    t, K, L = olat.pair_lags(T_obs, T_sft, T_max, Q)
    mu = 0.01
    lam = np.array([A_P, tasc, P])
    off = lam.copy()
    off[i] += math.sqrt(mu / g[i, i])

    def roemer(l):
        inj = synth.Injection(h0=1.0, f0=F, a_p=l[0], T_asc=l[1], P=l[2])
        return synth.orbital_roemer_delay(inj, l[1], t)

    dphi = 2 * math.pi * F * (roemer(off) - roemer(lam))      # template minus signal phase
    loss = np.mean(1.0 - np.cos(dphi[K] - dphi[L]))
    assert abs(loss / mu - 1.0) < 0.05, loss


def test_library_metric_and_lattice_match_oracle():
    import paper_1712_06515_gb300 as cc
    from paper_1712_06515_gb300 import _lib
    _lib.build()
    for (T_obs, T_sft, T_max, Q) in ((86400.0 * 3, 240.0, 1200.0, 2), (86400.0 * 20, 360.0, 3600.0, 3)):
        ref = olat.metric(T_obs, T_sft, T_max, Q, F, A_P, 5000.0, P)
        got = cc.metric(T_obs, T_sft, T_max, Q, F, A_P, 5000.0, P)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    g = olat.metric(86400.0 * 10, 360.0, 3600.0, 2, F, A_P, 5000.0, P)
    lo, hi = [1.36, 4000.0, P - 0.2], [1.52, 4600.0, P + 0.2]
    ref = olat.lattice(g, 0.1, lo, hi)
    got = cc.lattice(g, 0.1, lo, hi)
    np.testing.assert_array_equal(got, ref)


def test_library_metric_and_lattice_reject_bad_arguments():
    """Error behaviour of the host functions as the header states it: invalid sizes and
    ranges are CC_ERR_INVALID, an eccentric orbit is CC_ERR_UNSUPPORTED for the metric,
    and an output smaller than the lattice is refused after *n_out reports its size."""
    import ctypes
    import paper_1712_06515_gb300 as cc
    from paper_1712_06515_gb300 import _lib
    _lib.build()
    lib = _lib.load()
    dp = ctypes.POINTER(ctypes.c_double)
    orb = np.array([A_P, 5000.0, P, 0.0, 0.0])
    g = np.zeros(9)
    call = lambda T_obs, T_sft, T_max, Q, f, o: lib.crosscorr_metric(
        T_obs, T_sft, T_max, Q, f, o.ctypes.data_as(ctypes.c_void_p), 0.0, g.ctypes.data_as(dp))
    assert call(86400.0, 360.0, 3600.0, 2, F, orb) == 0
    assert call(86400.0, 0.0, 3600.0, 2, F, orb) == 1           # T_sft > 0
    assert call(86400.0, 360.0, -1.0, 2, F, orb) == 1           # T_max >= 0
    assert call(86400.0, 360.0, 3600.0, 0, F, orb) == 1         # 1 <= Q
    assert call(200.0, 360.0, 3600.0, 2, F, orb) == 1           # fewer than two SFTs
    ecc = orb.copy()
    ecc[3] = 0.2
    assert call(86400.0, 360.0, 3600.0, 2, F, ecc) == 5         # circular orbits only
    assert lib.crosscorr_metric(86400.0, 360.0, 3600.0, 2, F, None, 0.0, g.ctypes.data_as(dp)) == 1

    gm = olat.metric(86400.0 * 10, 360.0, 3600.0, 2, F, A_P, 5000.0, P).ravel().copy()
    lo = np.array([1.36, 4000.0, P - 0.2])
    hi = np.array([1.52, 4600.0, P + 0.2])
    n = ctypes.c_int64()
    args = lambda mu, l, h: (gm.ctypes.data_as(dp), mu, l.ctypes.data_as(dp), h.ctypes.data_as(dp))
    assert lib.crosscorr_lattice(*args(0.1, lo, hi), None, 0, ctypes.byref(n)) == 0 and n.value > 1
    small = np.zeros((n.value - 1, 5))
    assert lib.crosscorr_lattice(*args(0.1, lo, hi), small.ctypes.data_as(ctypes.c_void_p), n.value - 1,
                                 ctypes.byref(n)) == 1
    assert lib.crosscorr_lattice(*args(0.0, lo, hi), None, 0, ctypes.byref(n)) == 1      # mu > 0
    assert lib.crosscorr_lattice(*args(0.1, hi, lo), None, 0, ctypes.byref(n)) == 1      # lo <= hi
    with pytest.raises(cc.CrossCorrError):
        cc.lattice(gm.reshape(3, 3), -1.0, lo, hi)
