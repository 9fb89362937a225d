"""Parity of the persistent, TMA-fed spectrum + pair-sum kernel of the two-pass path
(coset length 4096 with whole segments: N_FFT = 32768 or 16384, N_s = 3600) against the
FP64 oracle, through the C ABI.

The workloads are the 120-day band's segment geometry (T_sft = 360 s, T_short = 3600 s)
on two weeks of data with long gaps, so that whole (detector, segment) transforms are
skipped and the bulk-copy pipeline jumps over them.  Tolerances as in the other parity
tests: 1e-4 max(1, max|rho|) (FP32), 1e-2 (BF16 storage).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1712_06515_gb300 as cc  # noqa: E402

DEV = torch.device("cuda:0")

BASE = dict(n_samples=3600 * 14, T_sft=360.0, T_max=3600.0, T_short=3600.0, f_band=0.1, f_h=150.0,
            duty=0.6, mean_lock_s=7200.0)
CASES = {
    "R1": dict(),
    "R1_Q1": dict(n_det=1),
    "R1_all_ordered": dict(pair_mode=2),
    "R0": dict(T_max=0.0),
    "R1_D16": dict(D=16),
    "R1_ragged": dict(n_samples=3600 * 14 + 1802),   # partial last segment dropped
    "R1_odd_Ns": dict(T_max=3599.0, T_short=3599.0),   # odd segment length: the older kernel
    "R1_Ns3000": dict(n_samples=3000 * 16, T_max=3000.0, T_short=3000.0),   # 16 does not divide N_s
    "R1_Ns2180": dict(n_samples=2180 * 20, T_max=2180.0, T_short=2180.0, T_sft=218.0),
}


def case(name, seed=41, n_templates=3):
    kw = dict(BASE)
    kw.update(CASES[name])
    return synth.tiny(seed=seed, n_templates=n_templates, **kw)


def assert_close(got, ref, tol):
    for t in range(ref.shape[0]):
        err = float(np.abs(got[t] - ref[t]).max())
        lim = tol * max(1.0, float(np.abs(ref[t]).max()))
        assert err <= lim, f"template {t}: max |drho| = {err:.3e} > {lim:.3e}"


@pytest.mark.parametrize("name", sorted(CASES))
def test_coset4096_parity(name):
    ds = case(name)
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        assert plan.info["L"] == 4096 and plan.search_path == cc.PATH_TWO_PASS
        x = torch.from_numpy(ds.x64).to(DEV)
        tm = torch.from_numpy(ds.templates).to(DEV)
        got = plan.search(x, tm).cpu().numpy().astype(np.float64)
        plan.check()
    assert_close(got, ref, 1e-4)


def test_coset4096_bf16_storage():
    ds = case("R1")
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets, store=cc.STORE_BF16) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        got = plan.search(x, torch.from_numpy(ds.templates).to(DEV)).cpu().numpy().astype(np.float64)
        plan.check()
    assert_close(got, ref, 1e-2)


FOLD = {
    # N_s = 8000 on 4096 positions (two folds, 16 cosets)
    "F2": dict(n_samples=8000 * 8, T_sft=400.0, T_max=8000.0, T_short=8000.0, f_band=0.05, f_h=150.0,
               duty=0.6, mean_lock_s=20000.0),
    # N_s = 36000 (nine folds, 64 cosets): the long-lag segment geometry
    "F9": dict(n_samples=36000 * 4, T_sft=360.0, T_max=36000.0, T_short=36000.0, f_band=0.02, f_h=150.0,
               duty=0.7, mean_lock_s=40000.0),
}


@pytest.mark.parametrize("name", sorted(FOLD))
def test_folded_segments_bf16(name):
    """Segments longer than the 4096-point transform (BF16 storage): the fold kernel's
    C-point DFT over the fold index, then the persistent kernel, against the oracle at the
    BF16 bar, and against the staged path (same storage) to a tighter bound."""
    ds = synth.tiny(seed=43, n_templates=2, **FOLD[name])
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets, store=cc.STORE_BF16) as plan:
        assert plan.info["L"] == 4096 and plan.info["N_s"] > 4096
        assert plan.search_path == cc.PATH_TWO_PASS
        x = torch.from_numpy(ds.x64).to(DEV)
        tm = torch.from_numpy(ds.templates).to(DEV)
        got = plan.search(x, tm).cpu().numpy().astype(np.float64)
        plan.check()
        plan.set_path(cc.PATH_STAGED)
        staged = plan.search(x, tm).cpu().numpy().astype(np.float64)
    assert_close(got, ref, 1e-2)
    assert_close(got, staged, 3e-3)


PADDED = {
    "L2048": dict(n_samples=1800 * 12, T_max=1800.0, T_short=1800.0),
    "L1024": dict(n_samples=900 * 24, T_max=900.0, T_short=900.0, T_sft=300.0),
    "L512": dict(n_samples=480 * 40, T_max=480.0, T_short=480.0, T_sft=240.0),
    "L2048_R0": dict(n_samples=2000 * 10, T_max=0.0, T_short=2000.0, T_sft=400.0),
    "L2048_Q1_all_ordered": dict(n_samples=1800 * 12, T_max=1800.0, T_short=1800.0, n_det=1, pair_mode=2),
}


@pytest.mark.parametrize("name", sorted(PADDED))
def test_shorter_cosets_padded_to_4096(name):
    """A plan whose own coset length is below 4096 (segments of at most 2048 samples) takes
    the persistent kernel's 4096-point cosets when tuned to (transform_len = 4096): the
    segments are zero-padded, fewer cosets cover the band.  Both tilings match the oracle."""
    kw = dict(BASE)
    kw.update(PADDED[name])
    ds = synth.tiny(seed=47, n_templates=3, **kw)
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        assert plan.info["L"] < 4096 <= plan.info["N_FFT"] and plan.search_path == cc.PATH_TWO_PASS
        x = torch.from_numpy(ds.x64).to(DEV)
        tm = torch.from_numpy(ds.templates).to(DEV)
        own = plan.search(x, tm).cpu().numpy().astype(np.float64)
        plan.set_tuning(transform_len=4096)
        padded = plan.search(x, tm).cpu().numpy().astype(np.float64)
        plan.check()
    assert_close(own, ref, 1e-4)
    assert_close(padded, ref, 1e-4)


def test_coset4096_loud_injection_topk():
    """A loud injection on a template of the batch: the top-10 (template, bin) list equals
    the oracle's."""
    probe = case("R1")
    p = oracle.make_plan(probe.cfg)
    tasc = synth.T_ASC_O1 + 20.0
    inj = synth.Injection(h0=0.5, f0=p.freq[700], a_p=1.44, T_asc=tasc, P=synth.SCO_X1_P, cosi=0.4)
    tm = np.array([[1.40, tasc - 150.0, synth.SCO_X1_P], [1.44, tasc, synth.SCO_X1_P],
                   [1.47, tasc + 90.0, synth.SCO_X1_P]])
    kw = dict(BASE)
    ds = synth.tiny(seed=41, injection=inj, templates=tm, **kw)
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        rho = plan.search(x, torch.from_numpy(tm).to(DEV))
        hits = plan.topk(rho, 10)
    assert_close(rho.cpu().numpy().astype(np.float64), ref, 1e-4)
    ti, bi, _ = oracle.topk(ref, 10)
    assert (hits["tmpl"][0], hits["bin"][0]) == (1, 700)
    assert list(zip(hits["tmpl"], hits["bin"])) == list(zip(ti, bi))


def test_coset4096_repeatable_and_split_independent():
    """Units are handed out dynamically, but each (template, weight, chunk, coset) unit is
    computed by one CTA in a fixed order: repeated runs give the same bits.  Other work
    splits (chunk counts) regroup the sums and agree with the staged path to rounding."""
    ds = case("R1", n_templates=5)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        tm = torch.from_numpy(ds.templates).to(DEV)
        runs = [plan.search(x, tm).cpu().numpy() for _ in range(3)]
        for r in runs[1:]:
            assert np.array_equal(r, runs[0])
        plan.set_path(cc.PATH_STAGED)
        staged = plan.search(x, tm).cpu().numpy()
        plan.set_path(cc.PATH_TWO_PASS)
        lim = 1e-5 * max(1.0, float(np.abs(staged).max()))
        for waves in (1, 3, 200):
            plan.set_tuning(chunk_waves=waves)
            got = plan.search(x, tm).cpu().numpy()
            assert np.abs(got - staged).max() <= lim, waves
        plan.check()


def test_bounded_wait_runs_out_reports_timeout_and_context_survives():
    """The persistent kernel bounds every wait on its bulk copies (about one second of
    clock).  With the wait test on, each CTA's first copy is never issued: the wait runs
    out, the CTA records it and returns, crosscorr_plan_check raises CC_ERR_TIMEOUT once,
    and the next search on the same context gives the same bits as before."""
    ds = case("R1")
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        tm = torch.from_numpy(ds.templates).to(DEV)
        good = plan.search(x, tm).cpu().numpy()
        plan.check()
        plan.set_wait_test(True)
        plan.search(x, tm)
        with pytest.raises(cc.CrossCorrError) as e:
            plan.check()
        assert e.value.status == 4   # CC_ERR_TIMEOUT
        plan.check()                 # the error word was cleared
        plan.set_wait_test(False)
        again = plan.search(x, tm).cpu().numpy()
        plan.check()
    assert np.array_equal(again, good)


@pytest.mark.parametrize("name,padded", [("R1", False), ("R1_Q1", False), ("R1_Ns3000", False),
                                         ("L2048", True)])
def test_staged_segment_fft_on_4096_cosets(name, padded):
    """The staged segment-FFT stage on 4096-point cosets (the persistent kernel writing
    spectra instead of pair sums; all-zero segments written as zeros without a transform):
    random series with some zero segments in, every spectrum bin against the oracle's
    zero-padded FP64 FFT route."""
    kw = dict(BASE)
    kw.update(CASES.get(name, PADDED.get(name, {})))
    ds = synth.tiny(seed=53, n_templates=2, **kw)
    p = oracle.make_plan(ds.cfg)
    assert ds.cfg.n_samples == p.M * p.N_s
    Q = ds.cfg.n_det
    rng = np.random.default_rng(7)
    a0 = rng.standard_normal((2, Q, 2, p.M * p.N_s)) + 1j * rng.standard_normal((2, Q, 2, p.M * p.N_s))
    for K in range(0, p.M, 3):   # some all-zero segments (as the resampling stage writes gaps)
        a0[K % 2, K % Q, (K // 3) % 2, K * p.N_s:(K + 1) * p.N_s] = 0
    r = np.arange(p.M * p.N_s)
    rot = np.exp(-2j * np.pi * ((p.f_r * r * p.dt) % 1.0))
    Fref = np.zeros((2, Q, p.M, 2, p.N_f), np.complex128)
    for t in range(2):
        for q in range(Q):
            for w in range(2):
                Fref[t, q, :, w] = oracle.spectra_fft(a0[t, q, w], p)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        assert (plan.info["L"] == 4096) != padded
        if padded:
            plan.set_tuning(transform_len=4096)
        ab = torch.from_numpy((a0 * rot).astype(np.complex64)).to(DEV)
        F = plan.segment_fft(ab, 2).cpu().numpy()
    err = np.abs(F - Fref).max()
    assert err <= 1e-5 * np.abs(Fref).max(), err


def test_staged_search_bf16_on_4096_cosets():
    """The staged path with BF16 storage on 4096-point cosets (the spectra mode reading
    bf16 pairs): against the oracle at the BF16 bar and against the two-pass path with the
    same storage to a tighter bound."""
    ds = case("R1")
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets, store=cc.STORE_BF16) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        tm = torch.from_numpy(ds.templates).to(DEV)
        plan.set_path(cc.PATH_STAGED)
        staged = plan.search(x, tm).cpu().numpy().astype(np.float64)
        plan.set_path(cc.PATH_TWO_PASS)
        two_pass = plan.search(x, tm).cpu().numpy().astype(np.float64)
        plan.check()
    assert_close(staged, ref, 1e-2)
    assert_close(staged, two_pass, 3e-3)
