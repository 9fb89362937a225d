"""FP64 evaluation of the learned 8-tap interpolator, for the oracle's resampler.

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the CPU
legs of bench.py.

The paper has no learned interpolator: it resamples with the 2D+1-tap windowed sinc
of Eq. shannon-interp-formula only.  The learned stand-in is a small network

    taps = W3^T tanh(W2^T tanh(W1^T s + b1) + b2) + b3,    s = (2u - 1, (2 nu_c - lo - hi)/(hi - lo)),

mapping the fractional sample offset u = t/dt' - floor(t/dt') and the band half-width
nu_c (cycles per sample) to 8 taps that multiply x_{floor(t/dt')-3} .. x_{floor(t/dt')+4}.
The weights file holds W1 [2,64], b1, W2 [64,64], b2, W3 [64,8], b3 (values exactly
representable in BF16), the range (lo, hi) of nu_c the inputs are scaled from and the
first tap's offset.  Evaluated here in FP64 straight from that definition.

PARITY UNPINNED against the paper (it has no such component).  What pins this code is
the mathematics of interpolation: a trained network must reproduce band-limited tones
to within its training error, which a transposed layer, a wrong activation, a wrong
tap offset or a wrong input scaling would destroy (tests/test_oracle_pins.py), and
its rho is judged against the exact D = 16 stencil.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class LearnedModel:
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray
    nu_lo: float
    nu_hi: float
    tap_offset: int

    @property
    def n_taps(self) -> int:
        return self.W3.shape[1]


def load(path: str) -> LearnedModel:
    z = np.load(path)
    if str(z["activation"]) != "tanh":
        raise ValueError("only tanh networks are defined")
    w = [np.asarray(z[k], np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    lo, hi = (float(v) for v in z["nu_c_range"])
    return LearnedModel(*w, nu_lo=lo, nu_hi=hi, tap_offset=int(z["tap_offset"]))


def taps(model: LearnedModel, u: np.ndarray, nu_c: float) -> np.ndarray:
    """Taps [..., 8] at offsets u in [0, 1) for band half-width nu_c."""
    u = np.asarray(u, np.float64)
    s = np.stack([2.0 * u - 1.0,
                  np.full_like(u, (2.0 * nu_c - model.nu_lo - model.nu_hi) / (model.nu_hi - model.nu_lo))], -1)
    h = np.tanh(s @ model.W1 + model.b1)
    h = np.tanh(h @ model.W2 + model.b2)
    return h @ model.W3 + model.b3


def interpolate(x: np.ndarray, jstar: np.ndarray, delta: np.ndarray, model: LearnedModel,
                nu_c: float) -> np.ndarray:
    """x(t) at t/dt' = j* + delta (delta in [-1/2, 1/2)) from the 8 samples around it:
    floor(t/dt') = j* (delta >= 0) or j* - 1, u = t/dt' - floor(t/dt').  Samples
    outside [0, N_t) are zero."""
    x = np.asarray(x)
    N_t = x.shape[0]
    jstar = np.asarray(jstar, np.int64)
    delta = np.asarray(delta, np.float64)
    neg = delta < 0
    j0 = np.where(neg, jstar - 1, jstar)
    u = np.where(neg, delta + 1.0, delta)
    c = taps(model, u, nu_c)
    acc = np.zeros(np.shape(delta), np.complex128)
    for n in range(model.n_taps):
        j = j0 - model.tap_offset + n
        ok = (j >= 0) & (j < N_t)
        acc += np.where(ok, x[np.clip(j, 0, N_t - 1)], 0.0) * c[..., n]
    return acc
