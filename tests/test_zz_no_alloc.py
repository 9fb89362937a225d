"""crosscorr_search_noalloc, the entry point for callers that cannot allocate device
memory during a search (for instance a service whose own pool owns all device memory
and forbids further cudaMalloc/cudaFree).  It must give crosscorr_search's result,
call after call, with its scratch taken from a fixed array inside the library.  This
file is collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1712_06515_gb300 as cc  # noqa: E402
from paper_1712_06515_gb300 import _lib  # noqa: E402

TOL32 = 1e-4   # the FP32 parity tolerance of the other GPU tests, relative to max(1, |rho|)


def _call_noalloc(lib, plan, x, tm, rho):
    xp = (ctypes.c_void_p * plan.Q)(*[int(x[i].data_ptr()) for i in range(plan.Q)])
    tm = cc.templates5(tm)
    st = lib.crosscorr_search_noalloc(plan._h, xp, int(tm.data_ptr()), tm.shape[0], int(rho.data_ptr()),
                                      int(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_search_matches_search_twice():
    lib = _lib.load()
    ds = synth.tiny(seed=77, n_templates=5,
                    injection=synth.Injection(h0=0.3, f0=120.11, a_p=1.44, T_asc=synth.T_ASC_O1,
                                              P=synth.SCO_X1_P))
    dev = torch.device("cuda:0")
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x = torch.from_numpy(ds.x64).to(dev)
        tm = torch.from_numpy(ds.templates).to(dev)
        ref = plan.search(x, tm).cpu().numpy().astype(np.float64)
        tol = TOL32 * max(1.0, float(np.abs(ref).max()))
        for _ in range(2):
            rho = torch.full((tm.shape[0], plan.N_f), np.nan, dtype=torch.float32, device=dev)
            assert _call_noalloc(lib, plan, x, tm, rho) == 0, lib.crosscorr_last_error()
            torch.cuda.synchronize()
            got = rho.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(got))
            assert float(np.abs(got - ref).max()) <= tol


def test_noalloc_rejects_oversized_batch():
    lib = _lib.load()
    ds = synth.tiny(seed=78, n_templates=1)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        xp = (ctypes.c_void_p * plan.Q)(*([None] * plan.Q))
        st = lib.crosscorr_search_noalloc(plan._h, xp, None, 65537, None, None)
        assert st == 1
        assert b"65536" in lib.crosscorr_last_error()
