"""Plain FP64 NumPy restatement of Appendix B: short Fourier transforms -> the
heterodyned, downsampled time series the resampled search starts from.

TEST INFRASTRUCTURE: imported only by tests/.

* SFT K covers [t_K - T_sft/2, t_K + T_sft/2) with t_K - T_sft/2 = K T_sft; its bins
  x~_Kk = sum_j x(t_K - T_sft/2 + j dt) exp(-2 pi i j k / N) dt (Eq. fourier-transform-def).
* The band of N' = Delta f_load T_sft bins centred on k_h = f_h T_sft (f_h on a bin,
  the remainder f_r being handled by the search's f_r*), inverse transformed with the
  half-band index shift m = l + N'/2, gives at the downsampled times j' dt'
  (dt' = T_sft / N')
      x_K,s(j') = (-1)^j' sum_{m<N'} exp(2 pi i j' m / N') x~_K(m + k_h - N'/2) / T_sft
  (Eq. shifted-for-fft), and the series
      x^h(K T_sft + j' dt') = exp(-2 pi i f_h (t_K - T_sft/2)) x_K,s(j')
  (Eq. long-time-series-het-corrected), phase-aligned across SFTs; blocks without an
  SFT (gaps) are zero.
Times are relative to the series origin t0.
"""
from __future__ import annotations

import numpy as np


def series_from_sfts(band: np.ndarray, block_index: np.ndarray, n_blocks: int, T_sft: float,
                     f_h: float) -> np.ndarray:
    """band [n_sft][N']: SFT bins k_h - N'/2 .. k_h + N'/2 - 1 (DFT times dt);
    block_index [n_sft]: the T_sft block of each SFT.  Returns the complex series of
    n_blocks * N' samples at dt' = T_sft / N'."""
    band = np.asarray(band, np.complex128)
    n_sft, Np = band.shape
    j = np.arange(Np)
    out = np.zeros(n_blocks * Np, np.complex128)
    for s in range(n_sft):
        K = int(block_index[s])
        # N' * ifft = sum_m exp(+2 pi i j m / N') band[m]
        xs = np.where(j % 2 == 0, 1.0, -1.0) * np.fft.ifft(band[s]) * Np / T_sft
        cyc = f_h * (K * T_sft)
        cyc -= np.floor(cyc)
        out[K * Np:(K + 1) * Np] = np.exp(-2j * np.pi * cyc) * xs
    return out
