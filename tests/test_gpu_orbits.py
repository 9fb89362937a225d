"""Elliptical-orbit templates (Eqs. solve-for-E, Kepler-equation) on every CUDA path and in
the detector-frame statistic, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from oracle import demod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1712_06515_gb300 as cc  # noqa: E402

DEV = torch.device("cuda:0")
INJ = synth.Injection(h0=0.5, f0=120.1, a_p=1.44, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P, e=0.3, omega=1.1)
TM = np.array([[INJ.a_p, INJ.T_asc, INJ.P, INJ.e, INJ.omega],
               [INJ.a_p, INJ.T_asc, INJ.P, 0.0, 0.0],
               [1.40, INJ.T_asc + 120.0, INJ.P, 0.1, -2.0],
               [1.50, INJ.T_asc - 60.0, INJ.P, 0.6, 0.4]])


def dataset(**kw):
    return synth.tiny(seed=19, injection=INJ, templates=TM, **kw)


def assert_close(got, ref, tol):
    for t in range(ref.shape[0]):
        err = float(np.abs(got[t] - ref[t]).max())
        lim = tol * max(1.0, float(np.abs(ref[t]).max()))
        assert err <= lim, f"template {t}: max |drho| = {err:.3e} > {lim:.3e}"


@pytest.mark.parametrize("path", ["fused", "two_pass", "staged"])
def test_eccentric_search_parity(path):
    ds = dataset()
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        plan.set_path({"fused": cc.PATH_FUSED, "two_pass": cc.PATH_TWO_PASS, "staged": cc.PATH_STAGED}[path])
        got = plan.search(torch.from_numpy(ds.x64).to(DEV), torch.from_numpy(TM).to(DEV))
        got = got.cpu().numpy().astype(np.float64)
    assert_close(got, ref, 1e-4)
    assert int(got[0].argmax()) == int(ref[0].argmax())
    assert got[0].max() > got[1].max()


def test_eccentric_resample_stage_parity():
    ds = dataset()
    p = oracle.make_plan(ds.cfg)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        ab = plan.resample(torch.from_numpy(ds.x64).to(DEV), torch.from_numpy(TM).to(DEV))[0].cpu().numpy()
    r = np.arange(p.M * p.N_s)
    rot = np.exp(-2j * np.pi * ((p.f_r * r * p.dt) % 1.0))
    for t, tmpl in enumerate(TM):
        for q in range(ds.cfg.n_det):
            xr, js, de = oracle.resample(ds.x[q], ds.dets[q], ds.cfg, p, tmpl)
            al, be, _ = oracle.weights(ds.dets[q], ds.cfg, js, de)
            nsft = int(round(ds.cfg.T_sft / ds.cfg.dt))
            ok = ~((np.abs(de + 0.5) < 1e-5) | ((np.abs(de) < 1e-5) & (js % nsft == 0)))
            a = al * xr * rot
            assert np.abs(ab[t, q, 0] - a)[ok].max() <= 2e-5 * np.abs(a).max()


def test_eccentric_demod_parity():
    ds = dataset()
    ref = np.stack([demod.demod_rho(ds, t) for t in TM])
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        plan.demod_prepare(torch.from_numpy(ds.x64).to(DEV))
        got = plan.demod_search(torch.from_numpy(TM).to(DEV)).cpu().numpy().astype(np.float64)
    assert_close(got, ref, 1e-4)
