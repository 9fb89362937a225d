"""Pins of oracle/sft_series.py (Appendix B) against the definition of an SFT at the raw
sampling rate: raw-rate SFTs of a band-limited signal come back as its heterodyned,
downsampled samples, phase-continuous across SFTs, with zeros in gaps."""
import numpy as np
import pytest

from oracle import sft_series

T_SFT, N_PRIME, OVER = 64.0, 32, 8          # 32 samples at dt' = 2 s per SFT, raw rate 8x higher


def raw_sfts(raw_of_t, blocks, k_h):
    """SFT bins k_h - N'/2 .. k_h + N'/2 - 1 of a raw signal, from Eq. fourier-transform-def
    at the raw rate (N = OVER N' samples per SFT)."""
    N = OVER * N_PRIME
    dt = T_SFT / N
    out = []
    for K in blocks:
        t = K * T_SFT + dt * np.arange(N)
        xt = np.fft.fft(raw_of_t(t)) * dt          # sum_j x(t_s + j dt) exp(-2 pi i j k / N) dt
        k = (k_h + np.arange(-N_PRIME // 2, N_PRIME // 2)) % N
        out.append(xt[k])
    return np.array(out)


def test_round_trip_of_a_band_limited_series():
    rng = np.random.default_rng(4)
    n_blocks, k_h = 6, 96                      # f_h = k_h / T_sft = 1.5 Hz, on a bin
    f_h = k_h / T_SFT
    dtp = T_SFT / N_PRIME
    x = (rng.standard_normal(n_blocks * N_PRIME) + 1j * rng.standard_normal(n_blocks * N_PRIME))
    # the raw signal whose heterodyned samples are x: per block, the band-limited periodic
    # interpolation of the block's samples, shifted up by f_h
    X = np.fft.fft(x.reshape(n_blocks, N_PRIME), axis=1)
    l = np.fft.fftfreq(N_PRIME, 1.0 / N_PRIME)

    def raw(t):
        K = int(np.floor(t[0] / T_SFT))
        tau = t - K * T_SFT
        xh = (X[K][None, :] * np.exp(2j * np.pi * np.outer(tau, l) / T_SFT)).sum(1) / N_PRIME
        return xh * np.exp(2j * np.pi * f_h * t)

    blocks = np.arange(n_blocks)
    band = raw_sfts(raw, blocks, k_h)
    got = sft_series.series_from_sfts(band, blocks, n_blocks, T_SFT, f_h)
    np.testing.assert_allclose(got, x, rtol=0, atol=1e-10)
    assert abs(dtp - 2.0) < 1e-15


@pytest.mark.parametrize("k_h", [96, 97])       # odd k_h: f_h (K + 1/2) T_sft is not an integer
@pytest.mark.parametrize("dl", [5, -11, 0])
def test_tone_on_a_bin_is_phase_continuous_across_sfts(dl, k_h):
    f_h = k_h / T_SFT
    f = (k_h + dl) / T_SFT
    phi = 0.4
    blocks = np.array([0, 1, 2, 4, 5])           # block 3 is a gap
    band = raw_sfts(lambda t: 1.3 * np.exp(1j * (2 * np.pi * f * t + phi)), blocks, k_h)
    got = sft_series.series_from_sfts(band, blocks, 6, T_SFT, f_h)
    t = (T_SFT / N_PRIME) * np.arange(6 * N_PRIME)
    expect = 1.3 * np.exp(1j * (2 * np.pi * (f - f_h) * t + phi))
    expect[3 * N_PRIME:4 * N_PRIME] = 0.0
    np.testing.assert_allclose(got, expect, rtol=0, atol=1e-10)
