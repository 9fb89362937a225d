"""The timed CPU baseline of bench.py (a plain FP32 implementation of the same algorithm:
FP64 knot timing, FP32 windowed-sinc interpolation and weights, complex64 pocketfft
segment transforms, FP32 pair sums) agrees with the FP64 oracle at the FP32 bar:
per template max |rho_cpu32 - rho_oracle| <= 1e-4 max(1, max|rho_oracle|)."""
import numpy as np
import pytest

import bench
import oracle
import synth

CASES = {
    "default": dict(),
    "T_max0": dict(T_max=0.0, T_short=64.0, f_band=0.3),
    "R2": dict(T_max=256.0, T_short=128.0),
    "Q1": dict(n_det=1),
    "Q3": dict(n_det=3),
    "cross_only": dict(pair_mode=1),
    "all_ordered": dict(pair_mode=2),
    "D16": dict(D=16),
    "ragged": dict(n_samples=4096 + 77),
    "segment_3600": dict(n_samples=3600 * 8, T_sft=360.0, T_max=3600.0, T_short=3600.0, f_band=0.1,
                         f_h=150.0, duty=0.6, mean_lock_s=7200.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_cpu_fp32_matches_oracle(name):
    ds = synth.tiny(seed=23, n_templates=3, **CASES[name])
    ref = oracle.rho(ds)
    got = bench.cpu_fp32_rho(ds, ds.templates, threads=2).astype(np.float64)
    assert got.shape == ref.shape
    for t in range(ref.shape[0]):
        err = float(np.abs(got[t] - ref[t]).max())
        lim = 1e-4 * max(1.0, float(np.abs(ref[t]).max()))
        assert err <= lim, f"template {t}: {err:.3e} > {lim:.3e}"


def test_cpu_fp32_plan_matches_oracle_plan():
    for kw in CASES.values():
        ds = synth.tiny(seed=23, n_templates=1, **kw)
        p = oracle.make_plan(ds.cfg)
        q = bench._cpu_plan(ds.cfg)
        assert (q["N_s"], q["M"], q["R"], q["N"], q["N_f"]) == (p.N_s, p.M, p.R, p.N_FFT, p.N_f)
        assert np.array_equal(q["idx"], np.mod(p.kbar - p.N_FFT // 2, p.N_FFT))
        np.testing.assert_allclose(q["dfreq"], p.dfreq, rtol=0, atol=1e-12)
