"""Plain FP64 NumPy restatement of the parameter-space metric and the cubic template
lattice (Sec. III A: Eqs. phase-derivs-metric, metric-spacing-eq).

TEST INFRASTRUCTURE: imported only by tests/.

g_ij = 1/2 < d(Phi_K - Phi_L)/d lambda^i  d(Phi_K - Phi_L)/d lambda^j >_alpha over the pairs
alpha = KL of the statistic, for lambda = (a_p, T_asc, P) of a circular orbit and the
signal phase Phi(t) = 2 pi f (t_SSB - a_p sin(Omega (t_SSB - T_asc))), Omega = 2 pi / P:

  dPhi/da_p   = -2 pi f sin(psi),                     psi = Omega (t - T_asc),
  dPhi/dT_asc =  2 pi f a_p Omega cos(psi),
  dPhi/dP     =  2 pi f a_p Omega (t - T_asc) cos(psi) / P.

Readings:
M1. The pairs are those of the detector-frame statistic (reading D2): SFT mid-times
    t_K = (k + 1/2) T_sft of an unbroken run, every unordered pair of distinct SFTs of
    the Q detectors with |t_K - t_L| <= T_max; same-time pairs of different detectors
    enter with zero phase difference.  The Earth's Roemer delay is common to both
    members of a pair to the accuracy the metric needs and is left out.
M2. A cubic lattice per Eq. metric-spacing-eq, delta lambda_i = sqrt(mu / g_ii), from the
    low end of each range, covering the range.
"""
from __future__ import annotations

import math

import numpy as np


def pair_lags(T_obs: float, T_sft: float, T_max: float, Q: int):
    """Mid-times of the SFTs and the (K, L) index pairs of reading M1 (per detector
    pair the same time grid)."""
    n = int(T_obs // T_sft)
    t = (np.arange(n) + 0.5) * T_sft
    Rs = int(math.floor(T_max / T_sft + 1e-9))
    K, L = [], []
    for lag in range(0, Rs + 1):
        k = np.arange(n - lag)
        # detector pairs: lag 0 -> X < Y (Q(Q-1)/2); lag > 0 -> all Q^2 ordered (X, Y)
        mult = Q * (Q - 1) // 2 if lag == 0 else Q * Q
        for _ in range(mult):
            K.append(k)
            L.append(k + lag)
    return t, np.concatenate(K), np.concatenate(L)


def phase_derivatives(t: np.ndarray, f: float, a_p: float, T_asc_rel: float, P: float) -> np.ndarray:
    """[3][n]: dPhi/d(a_p, T_asc, P) at times t (relative to t0)."""
    Om = 2.0 * math.pi / P
    psi = Om * (t - T_asc_rel)
    c = np.cos(psi)
    return np.stack([-2.0 * math.pi * f * np.sin(psi),
                     2.0 * math.pi * f * a_p * Om * c,
                     2.0 * math.pi * f * a_p * Om * (t - T_asc_rel) * c / P])


def metric(T_obs: float, T_sft: float, T_max: float, Q: int, f: float, a_p: float, T_asc_rel: float,
           P: float) -> np.ndarray:
    """g [3][3] of Eq. phase-derivs-metric (reading M1)."""
    t, K, L = pair_lags(T_obs, T_sft, T_max, Q)
    d = phase_derivatives(t, f, a_p, T_asc_rel, P)
    dd = d[:, K] - d[:, L]
    return 0.5 * (dd @ dd.T) / dd.shape[1]


def lattice(g: np.ndarray, mu: float, lo, hi) -> np.ndarray:
    """Cubic lattice of Eq. metric-spacing-eq over [lo, hi] per dimension (reading M2):
    rows (a_p, T_asc, P)."""
    axes = []
    for i in range(3):
        d = math.sqrt(mu / g[i, i])
        n = int(math.floor((hi[i] - lo[i]) / d + 1e-9)) + 1
        pts = lo[i] + d * np.arange(n)
        if pts[-1] < hi[i] - 1e-12 * max(1.0, abs(hi[i])):
            pts = np.append(pts, lo[i] + d * n)
        axes.append(pts)
    A, T, PP = np.meshgrid(*axes, indexing="ij")
    return np.stack([A.ravel(), T.ravel(), PP.ravel()], axis=1)
