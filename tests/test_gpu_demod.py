"""The detector-frame ("demodulation") CrossCorr on the GPU, through the C ABI, against
the FP64 oracle (oracle/demod.py): per template max |drho| <= 1e-4 max(1, max|rho|).
Both pair sums are covered: the method's pair loop (the default) and the separable
window-sum form (crosscorr_plan_set_demod_form)."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import demod

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1712_06515_gb300 as cc  # noqa: E402
from paper_1712_06515_gb300 import _lib  # noqa: E402

DEV = torch.device("cuda:0")
TOL = 1e-4
INJ = synth.Injection(h0=0.4, f0=120.1, a_p=1.44, T_asc=synth.T_ASC_O1, P=synth.SCO_X1_P)


def assert_close(got, ref, tol=TOL):
    for t in range(ref.shape[0]):
        err = float(np.abs(got[t] - ref[t]).max())
        lim = tol * max(1.0, float(np.abs(ref[t]).max()))
        assert err <= lim, f"template {t}: max |drho| = {err:.3e} > {lim:.3e}"


def gpu_demod(ds, templates=None, separable=False):
    tm = ds.templates if templates is None else templates
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        plan.demod_prepare(x)
        plan.set_demod_form(separable)
        return plan.demod_search(torch.from_numpy(np.ascontiguousarray(tm)).to(DEV)).cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("kw", [dict(), dict(T_max=0.0, T_short=64.0), dict(T_max=256.0, T_short=128.0),
                                dict(n_det=1), dict(n_det=3), dict(n_samples=4096 + 77),
                                dict(T_sft=32.0, T_max=160.0, T_short=160.0),
                                # R_s = 32 lags: the separable form recomputes leaving blocks
                                dict(T_sft=16.0, T_max=512.0, T_short=512.0)])
@pytest.mark.parametrize("separable", [False, True], ids=["pairs", "separable"])
def test_demod_parity(kw, separable):
    ds = synth.tiny(seed=33, n_templates=3, injection=INJ, **kw)
    ref = np.stack([demod.demod_rho(ds, t) for t in ds.templates])
    got = gpu_demod(ds, separable=separable)
    assert got.shape == ref.shape
    assert_close(got, ref)


def test_demod_injection_argmax_matches_oracle():
    ds = synth.tiny(seed=41, n_templates=3, injection=INJ, noise=False)
    ref = np.stack([demod.demod_rho(ds, t) for t in ds.templates])
    got = gpu_demod(ds)
    assert_close(got, ref)
    assert np.unravel_index(got.argmax(), got.shape) == np.unravel_index(ref.argmax(), ref.shape)


@pytest.mark.parametrize("separable", [False, True], ids=["pairs", "separable"])
def test_demod_o1_band_30_days_injected_template(separable):
    """30 days of the O1-shaped band (T_sft = 360 s SFTs, T_max = 3600 s: ten SFT lags).
    The separable form's window sums run over 7200 blocks here, through many add/subtract
    steps between their exact recomputations."""
    ds = synth.o1_band(n_ap=1, n_tasc=1, days=30)
    inj = ds.injection
    tm = np.array([[inj.a_p, inj.T_asc, inj.P]])
    ref = np.stack([demod.demod_rho(ds, t) for t in tm])
    got = gpu_demod(ds, tm, separable=separable)
    assert_close(got, ref)
    assert int(got[0].argmax()) == int(ref[0].argmax())


@pytest.fixture(scope="module")
def o1_band_120d():
    ds = synth.o1_band(n_ap=1, n_tasc=1, days=120)
    return ds, demod.sfts(ds)


@pytest.mark.parametrize("separable", [False, True], ids=["pairs", "separable"])
def test_demod_o1_band_full_size_sampled_bins(o1_band_120d, separable):
    """The workload `bench.py --method demod` times: 120 days, 33134 locked SFTs, 12356 bins.
    The injected template and a neighbour on the GPU (every bin) against the oracle at 24
    evenly spaced bins and the five bins around the GPU's peak.  The oracle's largest value
    among those five sits at the GPU's peak."""
    from oracle import make_plan
    ds, sft_list = o1_band_120d
    inj = ds.injection
    tm = np.array([[inj.a_p, inj.T_asc, inj.P], [inj.a_p + 0.02, inj.T_asc + 60.0, inj.P]])
    got = gpu_demod(ds, tm, separable=separable)
    freq = make_plan(ds.cfg).freq
    n_f = len(freq)
    assert got.shape == (2, n_f)
    for t in range(2):
        k = int(np.argmax(got[t]))
        near = list(range(max(0, k - 2), min(n_f, k + 3)))
        idx = np.array(sorted(set(np.linspace(0, n_f - 1, 24).astype(int).tolist()) | set(near)))
        ref = demod.demod_rho(ds, tm[t], freqs=freq[idx], sft_list=sft_list)
        err = float(np.abs(got[t][idx] - ref).max())
        lim = 1e-4 * max(1.0, float(np.abs(ref).max()))
        assert err <= lim, f"template {t}: max |drho| = {err:.3e} > {lim:.3e}"
        ref_near = ref[np.searchsorted(idx, near)]
        assert near[int(np.argmax(ref_near))] == k


def test_demod_forms_agree_to_rounding():
    """Pair loop and separable form on the same plan: the same rho up to FP32 rounding
    (a bound ten times tighter than the oracle bar), including gaps and a ragged end."""
    ds = synth.tiny(seed=35, n_templates=4, injection=INJ, n_samples=8192 + 301, duty=0.6)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        tm = torch.from_numpy(ds.templates).to(DEV)
        plan.demod_prepare(x)
        pairs = plan.demod_search(tm).cpu().numpy().astype(np.float64)
        plan.set_demod_form(True)
        sep = plan.demod_search(tm).cpu().numpy().astype(np.float64)
    assert_close(sep, pairs, 1e-5)


def test_demod_argument_errors():
    ds = synth.tiny(seed=33, n_templates=1)
    lib = _lib.load()
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        tm = cc.templates5(torch.from_numpy(ds.templates).to(DEV))
        rho = torch.empty((1, plan.N_f), dtype=torch.float32, device=DEV)
        st = lib.crosscorr_demod_search(plan._h, ctypes.c_void_p(int(tm.data_ptr())), 1,
                                        ctypes.c_void_p(int(rho.data_ptr())), None)
        assert st == 1                          # not prepared
        assert lib.crosscorr_plan_set_demod_form(plan._h, 2) == 1   # unknown form
        x = torch.from_numpy(ds.x64).to(DEV)
        with pytest.raises(cc.CrossCorrError) as e:
            plan.demod_prepare(x, n_bin=3)
        assert e.value.status == 5
        with pytest.raises(cc.CrossCorrError) as e:
            plan.demod_prepare(x, doppler_max=0.5)
        assert e.value.status == 1
