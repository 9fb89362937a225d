"""The batched multi-band workload (32 bands over 20-250 Hz, T_max from 240 to 3600 s,
10 days at 60 % duty) run from one CUDA graph launch, against the FP64 oracle with two
templates per band; the learned 8-tap interpolator on the same workload against the exact
D = 16 stencil as judge.  Oracle runs use a spawned process pool (no fork after CUDA)."""
import numpy as np
import pytest

import multiband_oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1712_06515_gb300 as cc  # noqa: E402
from paper_1712_06515_gb300.multiband import MultiBandSearch  # noqa: E402

DEV = torch.device("cuda:0")
N_BANDS = 32
PER_BAND = 2


def _oracle_all(D=None):
    return multiband_oracle.oracle_all(N_BANDS, PER_BAND, D)


@pytest.fixture(scope="module")
def bands():
    out = []
    for ds in synth.multiband(max_templates=PER_BAND):
        out.append((ds.cfg, ds.dets, torch.from_numpy(ds.x64).to(DEV), torch.from_numpy(ds.templates).to(DEV)))
    return out


def test_multiband_graph_parity(bands):
    ref = _oracle_all()
    mb = MultiBandSearch(bands, tune=True, tune_templates=PER_BAND).capture()
    got = [r.cpu().numpy().astype(np.float64) for r in mb.run()]
    torch.cuda.synchronize()
    for b, (g, r) in enumerate(zip(got, ref)):
        assert g.shape == r.shape, b
        for t in range(r.shape[0]):
            err = float(np.abs(g[t] - r[t]).max())
            lim = 1e-4 * max(1.0, float(np.abs(r[t]).max()))
            assert err <= lim, f"band {b} template {t}: {err:.3e} > {lim:.3e}"
    # the bands' paths as the autotuner chose them
    assert all(t["path"] in (cc.PATH_TWO_PASS, cc.PATH_FUSED) for t in mb.tuning)
    mb.close()


def test_multiband_graph_replay_equals_eager(bands):
    mb = MultiBandSearch(bands, tune=False)
    eager = [r.clone() for r in mb.run()]
    mb.capture()
    first = [r.clone() for r in mb.run()]
    second = [r.clone() for r in mb.run()]
    torch.cuda.synchronize()
    for e, f, s in zip(eager, first, second):
        assert torch.equal(e, f) and torch.equal(f, s)
    mb.close()


def test_multiband_learned_judged_by_exact_d16(bands):
    """The learned-interpolation variant of the workload: every band's rho within 1e-2
    max(1, max|rho|) of the exact D = 16 stencil's."""
    judge = _oracle_all(D=16)
    mb = MultiBandSearch(bands, interp=cc.INTERP_LEARNED, tune=False).capture()
    got = [r.cpu().numpy().astype(np.float64) for r in mb.run()]
    for b, (g, r) in enumerate(zip(got, judge)):
        for t in range(r.shape[0]):
            err = float(np.abs(g[t] - r[t]).max())
            lim = 1e-2 * max(1.0, float(np.abs(r[t]).max()))
            assert err <= lim, f"band {b} template {t}: {err:.3e} > {lim:.3e}"
    mb.close()
