"""The synthetic workloads have the shapes the search is specified on (CPU only)."""
import numpy as np

import oracle
import synth


def test_multiband_bands_follow_the_recipe():
    total = 0
    for b in range(32):
        x = b / 31
        T = 60.0 * round(4.0 * 15.0 ** x)
        total += round(1e3 * 50.0 ** x)
        assert 240.0 <= T <= 3600.0
    assert 4.0e5 < total < 4.3e5
    ds = synth.multiband_band(31, max_templates=3)
    assert ds.cfg.f_h == 250.0 and ds.cfg.T_max == ds.cfg.T_short == ds.cfg.T_sft == 3600.0
    assert ds.cfg.n_samples == 864000 and ds.templates.shape == (3, 3)
    ds0 = synth.multiband_band(0, max_templates=3)
    assert ds0.cfg.f_h == 20.0 and ds0.cfg.T_max == 240.0
    p = oracle.make_plan(ds0.cfg)
    assert (p.R, p.N_FFT, p.N_f) == (1, 2048, 823)
    # duty cycle near 60 % and each band's own gap pattern
    for d in (ds, ds0):
        duty = np.mean([np.mean(det.sigma > 0) for det in d.dets])
        assert 0.4 < duty < 0.8
    again = synth.multiband_band(0, max_templates=3)
    assert np.array_equal(again.x64, ds0.x64) and np.array_equal(again.templates, ds0.templates)
