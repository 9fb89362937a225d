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
