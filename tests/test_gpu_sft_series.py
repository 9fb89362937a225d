"""Appendix B's SFT -> heterodyned, downsampled series on the GPU against the oracle."""
import numpy as np
import pytest

from oracle import sft_series

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1712_06515_gb300 as cc  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("n_prime,T_sft,f_h", [(360, 360.0, 150.0), (64, 64.0, 120.0), (1440, 1440.0, 99.5),
                                               (64, 64.0, 120.015625),    # odd heterodyne bin 7681
                                               (225, 225.0, 101.0), (750, 750.0, 88.0),   # radices 3 and 5
                                               (7, 7.0, 100.0), (1, 1.0, 100.0),          # direct DFT
                                               (12800, 1280.0, 150.0),    # the largest mixed-radix size
                                               (14400, 1440.0, 150.0)])   # too large for it: direct DFT
def test_sfts_to_series_matches_oracle(n_prime, T_sft, f_h):
    rng = np.random.default_rng(n_prime)
    n_blocks = 40
    present = rng.uniform(size=n_blocks) < 0.7
    block_sft = np.full(n_blocks, -1, np.int64)
    block_sft[present] = np.arange(present.sum())
    band = (rng.standard_normal((present.sum(), n_prime)) + 1j * rng.standard_normal((present.sum(), n_prime))) * 30
    ref = sft_series.series_from_sfts(band, np.nonzero(present)[0], n_blocks, T_sft, f_h)
    got = cc.sfts_to_series(torch.from_numpy(band.astype(np.complex64)).to(DEV),
                            torch.from_numpy(block_sft).to(DEV), T_sft, f_h).cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 2e-5 * scale
    assert np.all(got.reshape(n_blocks, n_prime)[~present] == 0)


def test_sfts_to_series_full_size_120_day_band():
    """The launch bench.py times: one detector of the 120-day band (28800 blocks of 360 s at
    1 s, the band's own lock pattern, 16864 SFTs), every output sample against the oracle."""
    import synth
    ds = synth.o1_band(seed=1002)
    nsft = int(round(ds.cfg.T_sft / ds.cfg.dt))
    n_blocks = ds.cfg.n_samples // nsft
    locked = np.asarray(ds.dets[0].sigma[:n_blocks]) > 0
    block_sft = np.full(n_blocks, -1, np.int64)
    block_sft[locked] = np.arange(int(locked.sum()))
    rng = np.random.default_rng(1002)
    band = rng.standard_normal((int(locked.sum()), nsft)) + 1j * rng.standard_normal((int(locked.sum()), nsft))
    ref = sft_series.series_from_sfts(band, np.nonzero(locked)[0], n_blocks, ds.cfg.T_sft, ds.cfg.f_h)
    got = cc.sfts_to_series(torch.from_numpy(band.astype(np.complex64)).to(DEV),
                            torch.from_numpy(block_sft).to(DEV), ds.cfg.T_sft, ds.cfg.f_h).cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
    assert np.all(got.reshape(n_blocks, nsft)[~locked] == 0)


@pytest.mark.parametrize("n_blocks", [1, 3, 1000])
def test_sfts_to_series_every_block_a_gap(n_blocks):
    """No locked SFT: zeros everywhere (an empty band), written into a buffer that held
    other values."""
    out = torch.full((n_blocks * 360,), 5 + 5j, dtype=torch.complex64, device=DEV)
    band = torch.empty((0, 360), dtype=torch.complex64, device=DEV)
    bsd = torch.full((n_blocks,), -1, dtype=torch.int64, device=DEV)
    got = cc.sfts_to_series(band, bsd, 360.0, 150.0, out=out).cpu().numpy()
    assert np.all(got == 0)


def test_sfts_to_series_repeatable():
    """Blocks are taken from a counter in whatever order the warps arrive, but each block is
    transformed by one warp in a fixed order: repeated calls give the same bits."""
    rng = np.random.default_rng(5)
    n_blocks, n_prime = 5000, 360
    present = rng.uniform(size=n_blocks) < 0.6
    block_sft = np.full(n_blocks, -1, np.int64)
    block_sft[present] = np.arange(present.sum())
    band = torch.from_numpy((rng.standard_normal((present.sum(), n_prime))
                             + 1j * rng.standard_normal((present.sum(), n_prime))).astype(np.complex64)).to(DEV)
    bsd = torch.from_numpy(block_sft).to(DEV)
    a = cc.sfts_to_series(band, bsd, 360.0, 150.0).cpu().numpy()
    b = cc.sfts_to_series(band, bsd, 360.0, 150.0).cpu().numpy()
    assert np.array_equal(a, b)
