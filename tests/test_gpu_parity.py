"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (per template, in units of rho's unit noise): |rho_gpu - rho_oracle|
<= 1e-4 max(1, max|rho_oracle|) for the FP32 path, 1e-2 for BF16 storage.  Stage
tests feed oracle inputs to one GPU stage and compare its output element by
element.  Samples whose stencil centre or noise block is decided by a tie
(|delta| within 1e-5 of 1/2, or of 0 on a block boundary) are excluded from the
per-sample comparisons: the two sides round the same real number in different
precision there.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import Injection

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1712_06515_gb300 as cc  # noqa: E402

DEV = torch.device("cuda:0")
TOL32 = 1e-4
TOL16 = 1e-2


def dev_inputs(ds):
    return (torch.from_numpy(ds.x64).to(DEV), torch.from_numpy(ds.templates).to(DEV))


def rho_tol(ref, tol=TOL32):
    return tol * max(1.0, float(np.abs(ref).max()))


def assert_rho_close(got, ref, tol=TOL32):
    for t in range(ref.shape[0]):
        err = float(np.abs(got[t] - ref[t]).max())
        lim = rho_tol(ref[t], tol)
        assert err <= lim, f"template {t}: max |drho| = {err:.3e} > {lim:.3e}"


def oracle_ab(ds, plan, tmpl, q, rotate=True):
    """Oracle a_r, b_r (with the f_r* rotation exp(-2 pi i f_r* tau_r) that stage 1
    applies, unless rotate=False), segment norms, and a mask of tie-free samples."""
    xr, js, de = oracle.resample(ds.x[q], ds.dets[q], ds.cfg, plan, tmpl)
    al, be, s2 = oracle.weights(ds.dets[q], ds.cfg, js, de)
    r = np.arange(plan.M * plan.N_s)
    rot = np.exp(-2j * np.pi * ((plan.f_r * r * plan.dt) % 1.0)) if rotate else 1.0
    nsft = int(round(ds.cfg.T_sft / ds.cfg.dt))
    tie = (np.abs(de + 0.5) < 1e-5) | ((np.abs(de) < 1e-5) & (js % nsft == 0))
    return al * xr * rot, be * xr * rot, oracle.segment_norms(al, be, s2, plan), ~tie


CASES = {
    "default": dict(),
    "T_max0": dict(T_max=0.0, T_short=64.0, f_band=0.3),
    "R2": dict(T_max=256.0, T_short=128.0),
    "fband_005": dict(f_band=0.05, T_max=256.0, T_short=256.0),
    "Q1": dict(n_det=1),
    "Q3": dict(n_det=3),
    "cross_only": dict(pair_mode=1),
    "all_ordered": dict(pair_mode=2),
    "D16": dict(D=16),
    "ragged": dict(n_samples=4096 + 77),
    "short_series": dict(n_samples=300, T_sft=32.0, T_max=64.0, T_short=64.0),
    # coset lengths 512 / 1024 / 2048: last FFT passes of radix 2 / 4 / 8
    "L512": dict(T_max=512.0, T_short=512.0),
    "L1024": dict(n_samples=8192, T_max=1024.0, T_short=1024.0),
    "L2048": dict(n_samples=16384, T_max=2048.0, T_short=2048.0),
    "L2048_cross_only": dict(n_samples=16384, T_max=2048.0, T_short=2048.0, pair_mode=1),
    "L1024_Q3": dict(n_samples=8192, T_max=1024.0, T_short=1024.0, n_det=3),
}


def case_ds(name, seed=21, n_templates=3, **extra):
    kw = dict(CASES[name])
    kw.update(extra)
    return synth.tiny(seed=seed, n_templates=n_templates, **kw)


@pytest.mark.parametrize("name", sorted(CASES))
def test_search_parity(name):
    ds = case_ds(name)
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, tm = dev_inputs(ds)
        got = plan.search(x, tm).cpu().numpy().astype(np.float64)
    assert got.shape == ref.shape
    assert_rho_close(got, ref)


@pytest.mark.parametrize("name", ["default", "T_max0", "Q1", "all_ordered", "ragged", "L512", "L2048"])
@pytest.mark.parametrize("path", ["fused", "two_pass", "staged"])
def test_search_paths_parity(name, path):
    """Every search path on plans that all three support, against the oracle."""
    ds = case_ds(name)
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        assert plan.search_path == cc.PATH_TWO_PASS
        plan.set_path({"fused": cc.PATH_FUSED, "two_pass": cc.PATH_TWO_PASS, "staged": cc.PATH_STAGED}[path])
        x, tm = dev_inputs(ds)
        got = plan.search(x, tm).cpu().numpy().astype(np.float64)
    assert_rho_close(got, ref)


def test_search_path_selection():
    with cc.CrossCorrPlan(case_ds("Q3").cfg, case_ds("Q3").dets) as plan:
        assert plan.search_path == cc.PATH_FUSED
        with pytest.raises(cc.CrossCorrError) as e:
            plan.set_path(cc.PATH_TWO_PASS)
        assert e.value.status == 5
        with pytest.raises(cc.CrossCorrError) as e:
            plan.set_path(7)
        assert e.value.status == 1
        plan.set_path(cc.PATH_STAGED)
        assert plan.search_path == cc.PATH_STAGED
    ds = case_ds("default")
    with cc.CrossCorrPlan(ds.cfg, ds.dets, store=cc.STORE_BF16) as plan:
        assert plan.search_path == cc.PATH_TWO_PASS
        with pytest.raises(cc.CrossCorrError) as e:
            plan.set_path(cc.PATH_FUSED)      # the fused kernel stores nothing: FP32 only
        assert e.value.status == 5


def test_plan_bins_match_oracle():
    for name in ("default", "fband_005", "T_max0"):
        ds = case_ds(name)
        p = oracle.make_plan(ds.cfg)
        with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
            assert np.array_equal(plan.kbar, p.kbar)
            np.testing.assert_allclose(plan.freqs, p.freq, rtol=0, atol=1e-12)
            for key, val in (("N_FFT", p.N_FFT), ("N_f", p.N_f), ("M", p.M), ("R", p.R),
                             ("N_s", p.N_s), ("k0", p.k0)):
                assert plan.info[key] == val, key
            assert plan.info["nu_R"] == p.nu_R and plan.info["f_r"] == p.f_r


@pytest.mark.parametrize("name", ["default", "fband_005", "ragged", "Q3"])
def test_resample_stage_parity(name):
    ds = case_ds(name)
    p = oracle.make_plan(ds.cfg)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, tm = dev_inputs(ds)
        ab, nrm = plan.resample(x, tm)
        ab = ab.cpu().numpy()
        nrm = nrm.cpu().numpy()
    for t, tmpl in enumerate(ds.templates):
        for q in range(ds.cfg.n_det):
            a, b, norms, ok = oracle_ab(ds, p, tmpl, q)
            scale = max(np.abs(a).max(), np.abs(b).max())
            assert ok.mean() > 0.999
            assert np.abs(ab[t, q, 0] - a)[ok].max() <= 2e-5 * scale
            assert np.abs(ab[t, q, 1] - b)[ok].max() <= 2e-5 * scale
            for i in range(3):
                np.testing.assert_allclose(nrm[t, q, :, i], norms[i], rtol=2e-5,
                                           atol=2e-5 * max(1e-30, np.abs(norms[i]).max()))


@pytest.mark.parametrize("ws_bytes", [256, None])
def test_resample_stage_knot_paths(ws_bytes):
    """The resampling stage takes its FP64 knots from the pre-pass when the workspace holds
    one template's knot records (zeros written where a detector's weights vanish over a
    segment) and computes them in each block when a caller-owned workspace is too small;
    both against the oracle, and against each other on the zeroed (detector, segment)s."""
    ds = case_ds("default", n_templates=2)
    p = oracle.make_plan(ds.cfg)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, tm = dev_inputs(ds)
        if ws_bytes is not None:
            plan.set_workspace(torch.empty(ws_bytes, dtype=torch.uint8, device=DEV))
        ab = torch.full((2, plan.Q, 2, plan.N_tau), float("nan"), dtype=torch.complex64, device=DEV)
        ab, nrm = plan.resample(x, tm, ab=ab)
        ab = ab.cpu().numpy()
        nrm = nrm.cpu().numpy()
    n_used = p.M * p.N_s
    for t, tmpl in enumerate(ds.templates):
        for q in range(ds.cfg.n_det):
            a, b, norms, ok = oracle_ab(ds, p, tmpl, q)
            assert np.isfinite(ab[t, q, :, :n_used]).all()      # every sample of every segment written
            scale = max(np.abs(a).max(), np.abs(b).max())
            assert np.abs(ab[t, q, 0, :n_used] - a)[ok].max() <= 2e-5 * scale
            assert np.abs(ab[t, q, 1, :n_used] - b)[ok].max() <= 2e-5 * scale
            dead = (nrm[t, q, :, 0] == 0) & (nrm[t, q, :, 1] == 0)
            for K in np.nonzero(dead)[0]:
                seg = slice(K * p.N_s, (K + 1) * p.N_s)
                assert np.all(ab[t, q, :, seg] == 0) and np.all(a[seg] == 0) and np.all(b[seg] == 0)


@pytest.mark.parametrize("name", ["default", "fband_005", "T_max0"])
def test_segment_fft_stage_parity(name):
    """Oracle a_r, b_r in, GPU spectra out, against the oracle's FFT route (which
    applies the f_r* rotation itself, so it gets the unrotated series)."""
    ds = case_ds(name, n_templates=2)
    p = oracle.make_plan(ds.cfg)
    Q = ds.cfg.n_det
    ab = np.zeros((2, Q, 2, p.M * p.N_s), np.complex64)
    Fref = np.zeros((2, Q, p.M, 2, p.N_f), np.complex128)
    for t, tmpl in enumerate(ds.templates):
        for q in range(Q):
            a, b, _, _ = oracle_ab(ds, p, tmpl, q)
            ab[t, q, 0], ab[t, q, 1] = a, b
            a0, b0, _, _ = oracle_ab(ds, p, tmpl, q, rotate=False)
            Fref[t, q, :, 0] = oracle.spectra_fft(a0, p)
            Fref[t, q, :, 1] = oracle.spectra_fft(b0, p)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        F = plan.segment_fft(torch.from_numpy(ab).to(DEV), 2).cpu().numpy()
    err = np.abs(F - Fref).max()
    assert err <= 1e-5 * np.abs(Fref).max(), err


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_pair_stage_parity(mode):
    """Oracle spectra and norms in, GPU rho out, against the oracle's pair sum."""
    ds = case_ds("R2", n_templates=2, n_det=3, pair_mode=mode)
    p = oracle.make_plan(ds.cfg)
    Q = ds.cfg.n_det
    F = np.zeros((2, Q, p.M, 2, p.N_f), np.complex64)
    nrm = np.zeros((2, Q, p.M, 4), np.float32)
    ref = np.zeros((2, p.N_f))
    rng = np.random.default_rng(5)
    for t in range(2):
        Fa = [(rng.standard_normal((p.M, p.N_f)) + 1j * rng.standard_normal((p.M, p.N_f))).astype(np.complex64)
              for _ in range(Q)]
        Fb = [(rng.standard_normal((p.M, p.N_f)) + 1j * rng.standard_normal((p.M, p.N_f))).astype(np.complex64)
              for _ in range(Q)]
        norms = [tuple(rng.uniform(0.5, 2.0, p.M).astype(np.float32) for _ in range(3)) for _ in range(Q)]
        for q in range(Q):
            F[t, q, :, 0], F[t, q, :, 1] = Fa[q], Fb[q]
            nrm[t, q, :, :3] = np.stack(norms[q], axis=1)
        Dn = oracle.normalization([tuple(n.astype(np.float64) for n in nq) for nq in norms], p, mode)
        raw = oracle.pair_sum([f.astype(np.complex128) for f in Fa], [f.astype(np.complex128) for f in Fb], p, mode)
        ref[t] = math.sqrt(2.0) * raw / math.sqrt(Dn)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        rho = plan.pair_accumulate(torch.from_numpy(F).to(DEV), torch.from_numpy(nrm).to(DEV), 2)
    assert_rho_close(rho.cpu().numpy().astype(np.float64), ref)


def test_staged_equals_search():
    ds = case_ds("default")
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, tm = dev_inputs(ds)
        ab, nrm = plan.resample(x, tm)
        F = plan.segment_fft(ab, tm.shape[0])
        staged = plan.pair_accumulate(F, nrm, tm.shape[0]).cpu().numpy()
        fused = plan.search(x, tm).cpu().numpy()
    assert_rho_close(fused.astype(np.float64), staged.astype(np.float64))


@pytest.mark.parametrize("path", ["two_pass", "staged"])
def test_bf16_storage_parity(path):
    ds = case_ds("default")
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets, store=cc.STORE_BF16) as plan:
        plan.set_path(cc.PATH_TWO_PASS if path == "two_pass" else cc.PATH_STAGED)
        x, tm = dev_inputs(ds)
        got = plan.search(x, tm).cpu().numpy().astype(np.float64)
    assert_rho_close(got, ref, TOL16)


def test_empty_and_degenerate_inputs():
    ds = case_ds("default")
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, tm = dev_inputs(ds)
        out = plan.search(x, tm[:0])
        assert out.shape == (0, plan.N_f)
        # a detector entirely in gaps contributes nothing; both in gaps gives rho = 0
        for d in ds.dets:
            d.sigma[:] = 0.0
        ds.x[:] = 0.0
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, tm = dev_inputs(ds)
        got = plan.search(x, tm).cpu().numpy()
    assert np.all(got == 0.0)
    np.testing.assert_array_equal(oracle.rho(ds), 0.0)


def test_bad_arguments_raise():
    ds = case_ds("default")
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, tm = dev_inputs(ds)
        with pytest.raises(ValueError):
            plan.search(x[:1], tm)
        with pytest.raises(ValueError):
            plan.search(x, tm.float())
        with pytest.raises(ValueError):
            plan.search(x.cpu(), tm)


def test_topk_matches_oracle_on_loud_injection():
    probe = synth.tiny(seed=31, noise=False)
    p = oracle.make_plan(probe.cfg)
    tasc = synth.T_ASC_O1 + 12.0
    inj = Injection(h0=0.6, f0=p.freq[150], a_p=1.44, T_asc=tasc, P=synth.SCO_X1_P, cosi=0.5)
    tm = np.array([[1.40, tasc, synth.SCO_X1_P], [1.44, tasc, synth.SCO_X1_P],
                   [1.44, tasc + 200.0, synth.SCO_X1_P], [1.48, tasc - 100, synth.SCO_X1_P]])
    ds = synth.tiny(seed=31, injection=inj, templates=tm)
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, t = dev_inputs(ds)
        rho = plan.search(x, t)
        hits = plan.topk(rho, 10)
    assert_rho_close(rho.cpu().numpy().astype(np.float64), ref)
    ti, bi, vi = oracle.topk(ref, 10)
    assert (hits["tmpl"][0], hits["bin"][0]) == (1, 150)
    assert list(zip(hits["tmpl"][:3], hits["bin"][:3])) == list(zip(ti[:3], bi[:3]))
    np.testing.assert_allclose(hits["rho"], vi, atol=rho_tol(ref))


def test_topk_ordering_and_ties():
    ds = case_ds("default")
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        vals = np.random.default_rng(3).standard_normal((7, plan.N_f)).astype(np.float32)
        vals[2, 5] = vals[0, 9] = vals[4, 1] = 9.0     # three-way tie at the top
        vals[6, 0] = np.nan                           # NaN never ranks
        rho = torch.from_numpy(vals).to(DEV)
        hits = plan.topk(rho, 20)
        ti, bi, vi = oracle.topk(np.nan_to_num(vals.astype(np.float64), nan=-np.inf), 20)
    assert list(zip(hits["tmpl"], hits["bin"])) == list(zip(ti, bi))
    assert list(zip(hits["tmpl"][:3], hits["bin"][:3])) == [(0, 9), (2, 5), (4, 1)]
    np.testing.assert_array_equal(hits["rho"], vi.astype(np.float32))
    assert np.allclose(hits["freq"], plan.freqs[hits["bin"]])


@pytest.mark.parametrize("kind,k", [("ramp", 4096), ("ramp", 700), ("normal", 4096), ("ties", 1000)])
def test_topk_many_tiles_per_block(kind, k):
    """Top-k over 2.5e7 values: each of the 304 pass-1 blocks scans ~160 tiles of 512.  A
    rising ramp admits every element of every tile, so candidate buffers fill and merge
    every few tiles with k near the buffer size; the result must equal the oracle's."""
    ds = case_ds("default")
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        n_t = -(-25_000_000 // plan.N_f)
        n = n_t * plan.N_f
        rng = np.random.default_rng(17)
        if kind == "ramp":
            vals = (np.arange(n, dtype=np.float64) * 1e-3 + rng.uniform(0, 5e-4, n)).astype(np.float32)
        elif kind == "normal":
            vals = rng.standard_normal(n).astype(np.float32)
        else:   # many equal values: ties decided by the flat index
            vals = rng.integers(0, 50, n).astype(np.float32)
        vals = vals.reshape(n_t, plan.N_f)
        hits = plan.topk(torch.from_numpy(vals).to(DEV), k)
        ti, bi, vi = oracle.topk(vals.astype(np.float64), k)
    assert list(zip(hits["tmpl"], hits["bin"])) == list(zip(ti, bi))
    np.testing.assert_array_equal(hits["rho"], vi.astype(np.float32))


def test_plain_day_all_templates():
    """One day, 1 Hz band at 100 Hz, 20% gaps, T_max = 0, the 4x4x4 grid (64 templates)."""
    ds = synth.plain_day()
    ref = oracle.rho(ds)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, tm = dev_inputs(ds)
        got = plan.search(x, tm).cpu().numpy().astype(np.float64)
    assert_rho_close(got, ref)


def test_plain_day_loud_injection_topk():
    probe = synth.plain_day(noise=False)
    p = oracle.make_plan(probe.cfg)
    ds = synth.plain_day(loudness=10.0, f0=p.freq[300])
    tm = ds.templates
    inj_t = int(np.argmin(np.abs(tm[:, 0] - 1.44) + np.abs(tm[:, 1] - ds.injection.T_asc)
                          + np.abs(tm[:, 2] - synth.SCO_X1_P)))
    sub = tm[[inj_t, 0, 21, 42, 63]]
    ref = oracle.rho(ds, templates=sub)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        rho = plan.search(x, torch.from_numpy(sub).to(DEV))
        hits = plan.topk(rho, 5)
    assert_rho_close(rho.cpu().numpy().astype(np.float64), ref)
    ti, bi, _ = oracle.topk(ref, 5)
    assert (ti[0], bi[0]) == (0, 300)
    assert list(zip(hits["tmpl"], hits["bin"])) == list(zip(ti, bi))


def test_o1_band_full_size_injected_template():
    """120 days, 60% duty, 0.5 Hz at 150 Hz, T_max = T_short = 3600 s: the full-size
    workload, checked on the injected template and one far template."""
    ds = synth.o1_band(n_ap=1, n_tasc=1)
    inj = ds.injection
    tm = np.array([[inj.a_p, inj.T_asc, inj.P], [1.52, inj.T_asc + 300.0, inj.P]])
    ref = oracle.rho(ds, templates=tm)
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        for path in (cc.PATH_TWO_PASS, cc.PATH_FUSED):
            plan.set_path(path)
            got = plan.search(x, torch.from_numpy(tm).to(DEV)).cpu().numpy().astype(np.float64)
            assert_rho_close(got, ref)


def test_o1_band_bench_launch_configuration_sampled_templates():
    """The launch configuration bench.py times, at full size: the first 80 templates of the
    8000-template grid (the bench's seed) in one search, i.e. two-pass batches of 72 and 8
    templates with the default 40-wave chunk split; the first and last template of each
    batch against the oracle at the FP32 bar."""
    ds = synth.o1_band()
    tm = np.ascontiguousarray(np.concatenate([ds.templates[:80], np.zeros((80, 2))], axis=1))
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        assert plan.search_path == cc.PATH_TWO_PASS
        x = torch.from_numpy(ds.x64).to(DEV)
        got = plan.search(x, torch.from_numpy(tm).to(DEV)).cpu().numpy().astype(np.float64)
    pick = [0, 71, 72, 79]
    ref = oracle.rho(ds, templates=ds.templates[pick])
    assert_rho_close(got[pick], ref)


def test_fused_search_is_deterministic_on_full_size_chunked_batch():
    """Race check: the fused kernel's halves and cluster peers meet only at barriers, so a
    chunked full-size batch (long gaps, segments with inactive detectors) gives the same
    bits every run and agrees with the staged path (no shared-memory hand-offs) to
    rounding, batched or one template at a time."""
    ds = synth.o1_band(n_ap=1, n_tasc=1)
    inj = ds.injection
    tm = np.array([[inj.a_p, inj.T_asc, inj.P], [1.40, inj.T_asc - 200.0, inj.P],
                   [1.52, inj.T_asc + 300.0, inj.P]])
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x = torch.from_numpy(ds.x64).to(DEV)
        tmd = torch.from_numpy(tm).to(DEV)
        ab, nrm = plan.resample(x, tmd)
        staged = plan.pair_accumulate(plan.segment_fft(ab, 3), nrm, 3).cpu().numpy()
        del ab, nrm
        lim = 1e-5 * max(1.0, float(np.abs(staged).max()))
        for path in (cc.PATH_FUSED, cc.PATH_TWO_PASS):
            plan.set_path(path)
            runs = [plan.search(x, tmd).cpu().numpy() for _ in range(3)]
            singles = np.stack([plan.search(x, tmd[i:i + 1]).cpu().numpy()[0] for i in range(3)])
            for r in runs[1:]:
                assert np.array_equal(r, runs[0]), path
            assert np.abs(runs[0] - staged).max() <= lim, path
            assert np.abs(singles - staged).max() <= lim, path


def test_fused_kernel_timing_events():
    ds = case_ds("default")
    with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
        x, tm = dev_inputs(ds)
        plan.search(x, tm)
        assert plan.kernel_time() == (0.0, 0)       # off by default
        plan.set_kernel_timing(True)
        plan.search(x, tm)
        plan.search(x, tm)
        plan.set_kernel_timing(False)
        plan.search(x, tm)
        ms, n = plan.kernel_time()
        assert n == 2 and ms > 0.0
        assert plan.kernel_time() == (0.0, 0)       # cleared by the read


def test_o1_band_long_lag_full_size():
    """The long-lag precision variant: T_max = T_short = 36000 s (N_FFT = 2^18, coset
    length 4096 with 36000 samples folded onto it, 123564 bins), the injected template.
    FP32 storage at the FP32 bar, BF16 storage of the resampled series at the BF16 bar;
    the per-template error is printed for the record."""
    ds = synth.o1_band(T_max=36000.0, n_ap=1, n_tasc=1)
    inj = ds.injection
    tm = np.array([[inj.a_p, inj.T_asc, inj.P]])
    ref = oracle.rho(ds, templates=tm)
    x = torch.from_numpy(ds.x64).to(DEV)
    tmd = torch.from_numpy(tm).to(DEV)
    for store, path, tol in ((cc.STORE_FP32, cc.PATH_TWO_PASS, TOL32), (cc.STORE_BF16, cc.PATH_TWO_PASS, TOL16),
                             (cc.STORE_BF16, cc.PATH_STAGED, TOL16)):
        with cc.CrossCorrPlan(ds.cfg, ds.dets, store=store) as plan:
            assert plan.info["L"] == 4096 and plan.info["N_FFT"] == 262144
            plan.set_path(path)
            got = plan.search(x, tmd).cpu().numpy().astype(np.float64)
        err = np.abs(got - ref).max(axis=1)
        print(f"store {store} path {path}: max|rho| {np.abs(ref).max():.2f}, per-template max error {err}")
        assert_rho_close(got, ref, tol)
        assert int(got[0].argmax()) == int(ref[0].argmax())
