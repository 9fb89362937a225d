"""Learned 8-tap interpolation weights: training and file I/O.

The resampler's exact interpolator is the 2D+1-tap windowed sinc.  The learned
variant replaces it by an 8-tap filter whose taps come from a small MLP

    (u, nu_c) -> 64 -> 64 -> 8 taps,   tanh between layers,

where u = t/dt - floor(t/dt) is the fractional sample offset and nu_c the half-width
(cycles per sample) of the band the series carries -- the local spectral context
(search half-band plus Doppler wings); both enter scaled to [-1, 1] by features().  The taps multiply x[floor(t)-3 .. floor(t)+4].
Weights are stored in BF16 and the network is evaluated with FP32 accumulation; the
training forward pass already uses the BF16-rounded weights (gradients pass straight
through the rounding), so the stored network is the one that was fitted.

Training data are windows of band-limited complex series of the kind the method
resamples (32 tones drawn uniformly in [-nu_c, nu_c], random amplitudes and phases)
with the exact value of the series at the offset as target; the MLP learns the
least-squares optimal taps for each (u, nu_c).  Run
`python -m paper_1712_06515_gb300.learned_interp` to regenerate
`learned_interp_weights.npz` (about three minutes on 4 CPU cores; identical up to the
order of floating-point reductions).  At nu_c = 0.2875 the stored network's error on
band-limited tones is 4.1e-3 at most and 8.4e-4 rms, against 1.2e-2 and 4.5e-3 for the
17-tap windowed sinc (D = 8).  This module is offline tooling: the search itself only
reads the weight file.
"""
from __future__ import annotations

import math
import os

import numpy as np

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "learned_interp_weights.npz")
IN_DIM, WIDTH, N_TAPS = 2, 64, 8
TAP_OFFSET = 3          # taps start at floor(t) - 3


def band_halfwidth(f_band: float, f_h: float, dt: float) -> float:
    """nu_c: half-width of the data's band in cycles/sample -- the searched half-band
    plus Doppler wings of 2.5e-4 f_h (Earth orbit ~1e-4, Sco X-1's orbit ~1.3e-4)."""
    return float(min(0.5, dt * (0.5 * f_band + 2.5e-4 * f_h)))


def to_bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 (round half to even), as float32."""
    a = np.ascontiguousarray(a, np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    rnd = ((bits >> 16) & 1) + 0x7FFF
    out = ((bits + rnd) >> 16).astype(np.uint32) << 16
    return out.astype(np.uint32).view(np.float32).reshape(a.shape)


def load_weights(path: str = WEIGHTS):
    """(W1 [2,64], b1, W2 [64,64], b2, W3 [64,8], b3) as BF16-exact float32 arrays."""
    z = np.load(path)
    return [z[k].astype(np.float32) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]


def flat_bf16_bits(weights) -> np.ndarray:
    """All layers concatenated (W1, b1, W2, b2, W3, b3, row-major) as BF16 bit patterns."""
    flat = np.concatenate([np.asarray(w, np.float32).ravel() for w in weights])
    return (to_bf16(flat).view(np.uint32) >> 16).astype(np.uint16)


NU_C_RANGE = (0.15, 0.32)   # band half-widths the network is trained for (0.5 Hz bands, 20-250 Hz)


def features(u, nu_c):
    """Network inputs scaled to [-1, 1]: the offset u in [0, 1) and nu_c in NU_C_RANGE."""
    lo, hi = NU_C_RANGE
    return np.stack([2.0 * np.asarray(u) - 1.0, (2.0 * np.asarray(nu_c) - (lo + hi)) / (hi - lo)], -1)


def _windows(n: int, rng: np.random.Generator, n_tones: int = 32):
    nu_c = rng.uniform(*NU_C_RANGE, n)
    u = rng.uniform(0.0, 1.0, n)
    # tone frequencies uniform on [-nu_c, nu_c], as a signal may sit anywhere in the band
    nu = rng.uniform(-1.0, 1.0, (n, n_tones)) * nu_c[:, None]
    amp = (rng.standard_normal((n, n_tones)) + 1j * rng.standard_normal((n, n_tones))) / math.sqrt(2 * n_tones)
    j = np.arange(N_TAPS) - TAP_OFFSET
    x = np.einsum("nk,nkj->nj", amp, np.exp(2j * np.pi * nu[:, :, None] * j[None, None, :]))
    y = np.einsum("nk,nk->n", amp, np.exp(2j * np.pi * nu * u[:, None]))
    return u, nu_c, x, y


def train(n_windows: int = 1_000_000, epochs: int = 300, seed: int = 1005, verbose: bool = True):
    import torch
    rng = np.random.default_rng(seed)
    u, nu_c, x, y = _windows(n_windows, rng)
    feats = torch.tensor(features(u, nu_c), dtype=torch.float32)
    xr = torch.tensor(np.stack([x.real, x.imag], -1), dtype=torch.float32)
    yr = torch.tensor(np.stack([y.real, y.imag], -1), dtype=torch.float32)
    torch.manual_seed(seed)
    net = torch.nn.Sequential(torch.nn.Linear(IN_DIM, WIDTH), torch.nn.Tanh(),
                              torch.nn.Linear(WIDTH, WIDTH), torch.nn.Tanh(),
                              torch.nn.Linear(WIDTH, N_TAPS))
    opt = torch.optim.Adam(net.parameters(), lr=2e-3)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=epochs)
    bs = 8192

    def bf16(w):
        # forward with the BF16-rounded weights the search will use, gradient straight through
        return w + (w.to(torch.bfloat16).to(torch.float32) - w).detach()

    def forward(f):
        h = torch.tanh(f @ bf16(net[0].weight).T + bf16(net[0].bias))
        h = torch.tanh(h @ bf16(net[2].weight).T + bf16(net[2].bias))
        return h @ bf16(net[4].weight).T + bf16(net[4].bias)

    for ep in range(epochs):
        perm = torch.randperm(n_windows)
        tot = 0.0
        for i in range(0, n_windows, bs):
            idx = perm[i:i + bs]
            c = forward(feats[idx])                               # [b, 8] real taps
            pred = torch.einsum("bn,bnc->bc", c, xr[idx])
            loss = ((pred - yr[idx]) ** 2).sum(-1).mean()
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += float(loss.detach()) * len(idx)
        sched.step()
        if verbose:
            print(f"epoch {ep}: mse {tot / n_windows:.3e}")
    Ws = [net[0].weight.T, net[0].bias, net[2].weight.T, net[2].bias, net[4].weight.T, net[4].bias]
    return [to_bf16(w.detach().numpy()) for w in Ws]


def save_weights(weights, path: str = WEIGHTS) -> None:
    """Weights plus the model definition a reader needs: the nu_c scaling range, the
    first tap's offset from floor(t) and the activation."""
    np.savez(path, **dict(zip(("W1", "b1", "W2", "b2", "W3", "b3"), weights)),
             nu_c_range=np.array(NU_C_RANGE, np.float64), tap_offset=np.array(TAP_OFFSET),
             activation=np.array("tanh"))


if __name__ == "__main__":
    import torch
    torch.set_num_threads(4)
    save_weights(train())
    print("wrote", WEIGHTS)
