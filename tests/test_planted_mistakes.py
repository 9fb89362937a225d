"""Mistakes planted in the oracle, on the CPU, each caught by its pins.

Every entry is a plausible error in the oracle's arithmetic (a sign, a dropped term, an
index or rounding slip, a transposed operand, a wrong scaling).  The test writes it into
the oracle module's source held in memory, executes that source in place of the module in
a fresh interpreter, re-binds the package's names to the mutated functions, and runs the
module's pin tests there: they must fail.  Nothing is written to disk.  An entry whose
text no longer occurs in the source fails the test, so the list follows the oracle.

Only mistakes that change some result are listed: with f_h on an SFT bin (the reading
the SFT-to-series conversion rests on) the per-SFT heterodyne factor exp(-2 pi i f_h K
T_sft) is exactly 1, so flipping its sign changes nothing and is not a mistake to catch.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUNNER = r"""
import importlib, sys
root, mod_name, path, old, new, pins = sys.argv[1:7]
sys.path.insert(0, root)
import oracle
mod = importlib.import_module(mod_name)
src = open(path).read()
if src.count(old) != 1:
    sys.exit(3)                                   # the planted text must occur exactly once
exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
for name in list(vars(oracle)):                   # the package re-exports the module's names
    obj = getattr(oracle, name)
    if getattr(obj, "__module__", None) == mod_name and name in mod.__dict__:
        setattr(oracle, name, mod.__dict__[name])
import pytest
sys.exit(10 + pytest.main([pins, "-x", "-q", "-p", "no:cacheprovider"]))
"""

CROSSCORR = [
    ("heterodyne sign", "return xi * np.exp(-2j * np.pi * cyc), jstar, delta",
     "return xi * np.exp(2j * np.pi * cyc), jstar, delta"),
    ("segment phase dropped", "        out[K] = Y[idx] * np.exp(-2j * np.pi * cyc)", "        out[K] = Y[idx]"),
    ("window shifted", "return 0.54 - 0.46 * np.cos(2.0 * np.pi * n / (2 * D))",
     "return 0.54 - 0.46 * np.cos(2.0 * np.pi * (n+0.5) / (2 * D+1))"),
    ("stencil rounding", "    g = 0.5 - np.asarray(e, np.float64)", "    g = 0.0 - np.asarray(e, np.float64)"),
    ("binary delay sign", "        return a_p * np.sin(2.0 * np.pi * ((u - tasc_rel) / P))",
     "        return -a_p * np.sin(2.0 * np.pi * ((u - tasc_rel) / P))"),
    ("C term dropped", "tot += A1 * A2 + B1 * B2 + 2.0 * C1 * C2", "tot += A1 * A2 + B1 * B2"),
    ("auto-pairs admitted", "elif X == Y and mode == PAIR_UNORDERED and 1 <= L - K:",
     "elif X == Y and mode == PAIR_UNORDERED and 0 <= L - K:"),
    ("conjugate missing", "acc += (np.conj(Fa[X][K]) * Fa[Y][L] + np.conj(Fb[X][K]) * Fb[Y][L]).real",
     "acc += (Fa[X][K] * Fa[Y][L] + np.conj(Fb[X][K]) * Fb[Y][L]).real"),
    ("f_r* sign", "f_r = paper_remainder(-cfg.f_band / 2.0, 1.0 / T_FFT)",
     "f_r = -paper_remainder(-cfg.f_band / 2.0, 1.0 / T_FFT)"),
    ("SSB delay sign", "        dl = ssb_delay(det, (tau + b) - dl)", "        dl = ssb_delay(det, (tau + b) + dl)"),
    ("weights at the wrong time", "    t = (jstar + delta) * cfg.dt\n", "    t = (jstar + 0*delta) * cfg.dt + 300\n"),
    ("bins rounded up", "kbar = k0 + np.floor(nu_R * k).astype(np.int64)",
     "kbar = k0 + np.ceil(nu_R * k).astype(np.int64)"),
    ("sigma for sigma^2", "    alpha = np.where(m, a / s2, 0.0)", "    alpha = np.where(m, a / np.sqrt(s2), 0.0)"),
    ("T_coh without 2 T_max", "T_coh = 2.0 * cfg.T_max + T_short", "T_coh = cfg.T_max + T_short"),
    ("metric spacing constant", "dlf = math.sqrt(6.0 * cfg.mu_f / math.pi) / T_coh",
     "dlf = math.sqrt(3.0 * cfg.mu_f / math.pi) / T_coh"),
    ("k0 one bin low", "f_FFT) * T_FFT + 1e-9))", "f_FFT) * T_FFT - 1e-9))"),
    ("f_FFT without the half band", "f_FFT = cfg.f_h + f_r - 0.5 / dt", "f_FFT = cfg.f_h + f_r"),
    ("taps mirrored", "acc += xj * (w[n] * np.sinc(delta - (n - D)))", "acc += xj * (w[n] * np.sinc(delta + (n - D)))"),
    ("table fraction reversed", "    f = u - i\n", "    f = i - u + 1.0\n"),
    ("noise-block tie", "return np.where((rem == 0) & (delta < 0), q - 1, q)",
     "return np.where((rem == 0) & (delta > 0), q - 1, q)"),
    ("b from the a table", "    b = _lerp(det.ab_t0, det.ab_dt, det.b_tab, t)", "    b = _lerp(det.ab_t0, det.ab_dt, det.a_tab, t)"),
    ("f_r* rotation sign", "pre = np.exp(-2j * np.pi * (plan.f_r * s * plan.dt))",
     "pre = np.exp(2j * np.pi * (plan.f_r * s * plan.dt))"),
    ("sqrt(2) dropped", "rho_k = math.sqrt(2.0) * raw / math.sqrt(Dn)", "rho_k = raw / math.sqrt(Dn)"),
    ("R rounded up", "R = int(math.floor(cfg.T_max / T_short + 1e-9))", "R = int(math.ceil(cfg.T_max / T_short + 1e-9))"),
    ("ragged tail kept", "M = int(cfg.n_samples) // N_s", "M = -(-int(cfg.n_samples) // N_s)"),
    ("remainder as printed (no final |b|)", "math.floor(abs(a) / abs(b)) * abs(b)", "math.floor(abs(a) / abs(b))"),
    ("direct DFT at absolute frequencies", "cyc = np.outer(plan.dfreq, r * plan.dt)", "cyc = np.outer(plan.freq, r * plan.dt)"),
    ("hat-A with sigma", "A = (alpha[:n] ** 2 * s2[:n])", "A = (alpha[:n] ** 2 * np.sqrt(s2[:n]))"),
    ("top-k ties by descending index", "order = np.lexsort((np.arange(flat.size), -flat))[:k]",
     "order = np.lexsort((-np.arange(flat.size), -flat))[:k]"),
]

DEMOD = [
    ("alternating sign dropped", "sign = np.where(m % 2 == 0, 1.0, -1.0)", "sign = 1.0"),
    ("conjugate missing", "raw += g * 2.0 * np.real(np.conj(Y[K]) * Y[L])", "raw += g * 2.0 * np.real(Y[K] * Y[L])"),
    ("phase sign", "Y.append(xi * zK * np.exp(-2j * np.pi * cyc))", "Y.append(xi * zK * np.exp(2j * np.pi * cyc))"),
    ("Doppler shift of the bin dropped", "x = (np.outer(dtau - 1.0, f) + dfreq[None, :]) * cfg.T_sft",
     "x = (0.0 * np.outer(dtau - 1.0, f) + dfreq[None, :]) * cfg.T_sft"),
    ("Xi dropped from N", "den += (XI[K] * XI[L] * g) ** 2", "den += (g) ** 2"),
    ("S_K without 2 dt", "        S = 2.0 * sig * sig * cfg.dt\n        z = xt", "        S = sig * sig\n        z = xt"),
    ("bins off by one", "m0 = np.floor(x).astype(np.int64) - (n_bin // 2 - 1)",
     "m0 = np.floor(x).astype(np.int64) - (n_bin // 2 - 1) + 1"),
    ("SFT start for its mid-time", "tmid = (ks * N + 0.5 * N) * cfg.dt", "tmid = (ks * N) * cfg.dt"),
    ("auto-pairs admitted", "for L in range(K + 1, n):", "for L in range(K, n):"),
    ("Xi weight dropped", "Y.append(xi * zK * np.exp(-2j * np.pi * cyc))", "Y.append(zK * np.exp(-2j * np.pi * cyc))"),
    ("b from the a table", "BH.append(scale * _lerp(det.ab_t0, det.ab_dt, det.b_tab, tmid))",
     "BH.append(scale * _lerp(det.ab_t0, det.ab_dt, det.a_tab, tmid))"),
    ("pairs at exactly T_max dropped", "if T[L] - T[K] > T_max + 1e-9:", "if T[L] - T[K] > T_max - 1e-9:"),
    ("2 dropped from the normalisation", "raw / np.sqrt(2.0 * den), 0.0)", "raw / np.sqrt(den), 0.0)"),
    ("Earth's Doppler dropped from dtau/dt", "return dl - R, (1.0 + ddl) * (1.0 - dR)", "return dl - R, (1.0 - dR)"),
    ("orbital Doppler sign", "return dl - R, (1.0 + ddl) * (1.0 - dR)", "return dl - R, (1.0 + ddl) * (1.0 + dR)"),
    ("(f - f_h) t dropped from the phase", "cyc = np.outer(d, f) + np.outer(tmid, dfreq)", "cyc = np.outer(d, f)"),
    ("z_K not divided by Xi", "return zK / xi, xi", "return zK, xi"),
    ("SSB slope per table step", "ddl = (det.ssb_delay[i + 1] - det.ssb_delay[i]) / det.eph_dt",
     "ddl = (det.ssb_delay[i + 1] - det.ssb_delay[i])"),
]

LEARNED = [
    ("W2 transposed", "h = np.tanh(h @ model.W2 + model.b2)", "h = np.tanh(h @ model.W2.T + model.b2)"),
    ("second activation dropped", "h = np.tanh(h @ model.W2 + model.b2)", "h = (h @ model.W2 + model.b2)"),
    ("tap offset", "j = j0 - model.tap_offset + n", "j = j0 - model.tap_offset + 1 + n"),
    ("u not scaled", "s = np.stack([2.0 * u - 1.0,", "s = np.stack([u,"),
    ("nu_c scaling", "(2.0 * nu_c - model.nu_lo - model.nu_hi)", "(nu_c - model.nu_lo - model.nu_hi)"),
    ("floor for negative offsets", "j0 = np.where(neg, jstar - 1, jstar)", "j0 = jstar"),
    ("u for negative offsets", "u = np.where(neg, delta + 1.0, delta)", "u = np.abs(delta)"),
    ("output bias dropped", "return h @ model.W3 + model.b3", "return h @ model.W3"),
    ("first bias dropped", "h = np.tanh(s @ model.W1 + model.b1)", "h = np.tanh(s @ model.W1)"),
    ("inputs swapped", "    h = np.tanh(s @ model.W1 + model.b1)", "    h = np.tanh(s[..., ::-1] @ model.W1 + model.b1)"),
    ("taps reversed", "acc += np.where(ok, x[np.clip(j, 0, N_t - 1)], 0.0) * c[..., n]",
     "acc += np.where(ok, x[np.clip(j, 0, N_t - 1)], 0.0) * c[..., model.n_taps - 1 - n]"),
    ("samples outside the series kept", "        ok = (j >= 0) & (j < N_t)\n        acc += np.where(ok,",
     "        ok = (j >= -N_t) & (j < N_t)\n        acc += np.where(ok,"),
]

ORBITS = [
    ("Kepler's equation sign", "dE = (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))",
     "dE = (E + e * np.sin(E) - M) / (1.0 - e * np.cos(E))"),
    ("periapsis from +w", "    nu = -omega", "    nu = omega"),
    ("cos E - e", "(np.cos(E) - e)", "(np.cos(E) + e)"),
    ("sqrt(1 - e^2) dropped", "math.sqrt(1.0 - e * e) * np.sin(E)", "(1.0 - e * e) * np.sin(E)"),
]

SFT_SERIES = [
    ("half-band sign dropped", "np.where(j % 2 == 0, 1.0, -1.0) * np.fft.ifft", "1.0 * np.fft.ifft"),
    ("heterodyne phase at the SFT mid-time", "cyc = f_h * (K * T_sft)", "cyc = f_h * ((K + 0.5) * T_sft)"),
    ("1/T_sft dropped", "* Np / T_sft", "* Np"),
]

LATTICE = [
    ("factor 1/2 dropped", "return 0.5 * (dd @ dd.T) / dd.shape[1]", "return (dd @ dd.T) / dd.shape[1]"),
    ("dPhi/dP without 1/P", "* (t - T_asc_rel) * c / P])", "* (t - T_asc_rel) * c])"),
    ("spacing mu / g", "d = math.sqrt(mu / g[i, i])", "d = mu / g[i, i]"),
    ("same-time pairs of one detector", "mult = Q * (Q - 1) // 2 if lag == 0 else Q * Q", "mult = Q * Q"),
    ("dPhi/da_p sign", "return np.stack([-2.0 * math.pi * f * np.sin(psi),",
     "return np.stack([2.0 * math.pi * f * np.sin(psi),"),
]

CASES = ([("oracle.crosscorr", "oracle/crosscorr.py", "tests/test_oracle_pins.py") + m for m in CROSSCORR]
         + [("oracle.crosscorr", "oracle/crosscorr.py", "tests/test_orbit_pins.py") + m for m in ORBITS]
         + [("oracle.sft_series", "oracle/sft_series.py", "tests/test_sft_series_pins.py") + m for m in SFT_SERIES]
         + [("oracle.lattice", "oracle/lattice.py", "tests/test_lattice.py") + m for m in LATTICE]
         + [("oracle.demod", "oracle/demod.py", "tests/test_demod_pins.py") + m for m in DEMOD]
         + [("oracle.learned", "oracle/learned.py", "tests/test_learned_pins.py") + m for m in LEARNED])


@pytest.mark.parametrize("mod_name,path,pins,what,old,new", CASES,
                         ids=[f"{os.path.basename(c[2])[:-3]}: {c[3]}" for c in CASES])
def test_planted_mistake_is_caught(mod_name, path, pins, what, old, new):
    r = subprocess.run([sys.executable, "-c", RUNNER, ROOT, mod_name, os.path.join(ROOT, path), old, new,
                        os.path.join(ROOT, pins)], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 3, f"{what}: the planted text is not in {path} (exactly once)"
    assert r.returncode >= 10, f"{what}: the runner failed\n{r.stdout[-1500:]}\n{r.stderr[-1500:]}"
    assert r.returncode != 10, f"{what}: planted in {path}, the pins of {pins} all passed"
