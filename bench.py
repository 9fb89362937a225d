"""Benchmark of the resampled CrossCorr search: rho template*frequency-bins per second.

Workload: 2 detectors, 120 days at 60% duty cycle in random lock segments, a
0.5 Hz band at 150 Hz sampled at 1 Hz (10,368,000 complex64 samples per
detector, 166 MB, larger than L2), T_sft = 360 s, T_max = T_short = 3600 s,
unit-variance Gaussian noise with an injected CW signal, and the orbital grid
a_p in [1.36, 1.52] lt-s (40) x T_asc +/- 300 s (200) with P fixed: 8000
templates x 12356 bins.  All inputs are synthetic (seeded), shaped like the
paper's Sco X-1 set-up.

One step is one pass of the whole path (resample -> segment spectra -> pair sum
-> normalised rho) over a batch of templates with the inputs resident in HBM.
Under torchrun each rank processes its own batch (weak scaling, no collective
on the data path); the max over ranks of the timed region sets the time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--templates B]
  python bench.py --impl reference      # the FP64 CPU oracle on a bounded sample
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CrossCorr rho templates*freq-bins/sec on 1 GB300 (+% HBM roofline) vs plain FP32 at stated rho error"
UNIT = "template*bins/s"
GRID_TEMPLATES = 8000
# DRAM bytes read + written per template by the spectrum kernel of this workload, from
# an ncu capture of one launch on 8 templates (its summary is kept with the profiles;
# the reads of a_r, b_r grow with the templates of a launch).  None once the kernel
# changes.
SEGPAIR_DRAM_BYTES_PER_TEMPLATE = (1.790227e9 + 46.770432e6) / 8
SM_COUNT = 152
FP32_LANES = 128
# days of the 120-day band in the bounded CPU samples (both CPU legs use the same sample)
CPU_SAMPLE_DAYS = 12.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--templates", type=int, default=GRID_TEMPLATES,
                    help="templates per step per rank (default: the whole 40x200 grid)")
    ap.add_argument("--path", default="search", choices=["search", "staged"])
    ap.add_argument("--workload", default="o1_band", choices=["o1_band", "o1_long", "multiband"],
                    help="o1_band: the 120-day single band (default); o1_long: the same band at "
                         "T_max = 36000 s with BF16 storage of the resampled series; multiband: 32 "
                         "bands over 20-250 Hz from one CUDA graph launch")
    ap.add_argument("--template-scale", type=float, default=0.25,
                    help="multiband: fraction of the 4.1e5-template grid per step")
    ap.add_argument("--method", default="resampled", choices=["resampled", "demod", "sft_series", "dft_gemm"],
                    help="resampled: the paper's method (default); demod: the detector-frame "
                         "statistic it replaces, on the same workload, for the speed comparison; "
                         "sft_series: the SFT-to-series input preparation of the 120-day band")
    ap.add_argument("--demod-form", default="pairs", choices=["pairs", "separable"],
                    help="demod: the method's pair loop (default) or the separable window-sum form")
    ap.add_argument("--pair-mode", default="unordered", choices=["unordered", "all_ordered"],
                    help="pair set: each unordered pair once (default) or every ordered pair with "
                         "auto-correlation (the F-statistic limit)")
    ap.add_argument("--eccentricity", type=float, default=0.0,
                    help="orbital eccentricity of every template (argument of periapsis 0.7 rad)")
    ap.add_argument("--interp", default="exact", choices=["exact", "learned"],
                    help="exact: windowed sinc, 2D+1 = 17 taps; learned: the 8-tap network")
    ap.add_argument("--search-path", default="auto", choices=["auto", "fused", "two_pass", "staged"],
                    help="force the path of crosscorr_search (auto: the library's choice)")
    ap.add_argument("--chunk-waves", type=int, default=0,
                    help="work split: target CTA waves of the segment-chunk split (0: library default)")
    ap.add_argument("--batch-templates", type=int, default=0,
                    help="work split: templates per two-pass batch (0: library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-days", type=float, default=CPU_SAMPLE_DAYS,
                    help="days of data in the bounded CPU oracle sample (both CPU legs)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the variant measurements (stencils, long lag, multi-band) of the default run")
    ap.add_argument("--e2e-steps", type=int, default=1)
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_peak(cc, clk):
    """(peak TFLOP/s, how): the lower of the FP32 FMA throughput measured on this GPU now
    (the library's full-occupancy FMA-chain kernel) and the derived SM count x 128 FP32
    lanes x 2 flop x maximum SM clock."""
    clk_max = float((clk or {}).get("sm_max_mhz") or 2070.0)
    derived = SM_COUNT * FP32_LANES * 2 * clk_max * 1e6 / 1e12
    try:
        measured = cc.measure_fp32_peak()
    except Exception:   # noqa: BLE001 - reported, the derived figure stands
        measured = None
    if measured and measured < derived:
        return measured, (f"measured: {measured:.2f} TFLOP/s FP32 FMA throughput on this GPU "
                          f"(derived {derived:.2f}: {SM_COUNT} SMs x {FP32_LANES} lanes x 2 x {clk_max:g} MHz)")
    return derived, (f"derived: {SM_COUNT} SMs x {FP32_LANES} FP32 lanes x 2 flop x {clk_max:g} MHz"
                     + (f" (measured {measured:.2f})" if measured else ""))


def spectrum_kernel_name(info, bf16=False):
    """The two-pass path's spectrum + pair-sum kernel(s) for this plan's geometry (the
    event pair of the plan's kernel timing brackets all of them)."""
    if info["L"] == 4096 and info["N_s"] % 16 == 0 and info["R"] <= 1:
        if info["N_s"] <= 4096:
            return "segpair_tma_kernel"
        if bf16:   # folded segments: the persistent kernel's shared memory holds a BF16 stage
            return ("fold64_kernel + segpair_tma_kernel" if info["C"] == 64
                    else "fold_kernel + segpair_tma_kernel")
    return "segpair_grouped_kernel" if info["L"] <= 2048 else "segpair_kernel"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [int(r[1]) for r in rows]
        mx = int(rows[0][2])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_sample(days, seed=1002):
    """The FP64 oracle, as it stands, on one template over the first `days` of the
    workload; returns (seconds, template*bins processed scaled to the full 120 d)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle
    import synth
    ds = synth.o1_band(seed=seed, days=days, n_ap=1, n_tasc=1)
    t = time.perf_counter()
    rho = oracle.rho(ds)
    dt = time.perf_counter() - t
    units = rho.shape[0] * rho.shape[1] * (days / 120.0)
    return dt, units


def cpu_oracle_baseline(days, min_seconds=10.0):
    """The oracle on the bounded sample, repeated until about min_seconds of CPU work."""
    tot_t, tot_u, n = 0.0, 0.0, 0
    while tot_t < min_seconds or n == 0:
        dt, u = cpu_oracle_sample(days)
        tot_t += dt
        tot_u += u
        n += 1
    return tot_u / tot_t, tot_t, n


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_sample(args.cpu_days)
    tot_t, tot_u = 0.0, 0.0
    for _ in range(args.steps):
        dt, units = cpu_oracle_sample(args.cpu_days)
        tot_t += dt
        tot_u += units
    value = tot_u / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "ranks_seen": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "o1_band: 2 det, 120 d at 60% duty, 0.5 Hz at 150 Hz, T_max=T_short=3600 s",
                   "sample": f"1 template x 12356 bins over the first {args.cpu_days:g} d, scaled to 120 d"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                         "sample": f"1 template, first {args.cpu_days:g} of 120 days, linear in T_obs"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Timed CPU baseline: a plain FP32 implementation of the same algorithm on the host cores
# ---------------------------------------------------------------------------
CPU_KNOT = 128          # FP64 timing at knots every 128 samples, a cubic between them
CPU_SEG_CHUNK = 256     # segments processed together (bounds the working set per thread)


def _cpu_plan(cfg):
    """Plan quantities of Sec. III B 2-4 (FP64): segment length, pair window, metric
    resolution, zero-padded FFT size, decimation and output bins, with the same readings
    as the GPU plan (T_short = max(T_max, T_sft) unless given, floor for "lround", the
    remainder with its final |b|, f_FFT = f_h + f_r* - 1/(2 dt'))."""
    dt = float(cfg.dt)
    T_short = float(cfg.T_short) if cfg.T_short > 0 else max(float(cfg.T_max), float(cfg.T_sft))
    N_s = int(round(T_short / dt))
    R = int(math.floor(cfg.T_max / T_short + 1e-9))
    M = int(cfg.n_samples) // N_s
    T_coh = 2.0 * cfg.T_max + T_short
    dlf = math.sqrt(6.0 * cfg.mu_f / math.pi) / T_coh
    N0 = (1.0 / dt / dlf) * math.ceil(dlf * T_coh)
    N = 1
    while N < N0:
        N *= 2
    T_FFT = N * dt
    nu_R = dlf * dt * N
    N_f = int(math.floor(cfg.f_band / dlf))
    a, b = -cfg.f_band / 2.0, 1.0 / T_FFT
    f_r = 0.0 if a == 0.0 else a - math.copysign(1.0, a) * math.floor(abs(a) / b) * b
    f_FFT = cfg.f_h + f_r - 0.5 / dt
    k0 = int(math.floor((cfg.f_h - cfg.f_band / 2.0 - f_FFT) * T_FFT + 1e-9))
    kbar = k0 + np.floor(nu_R * np.arange(N_f)).astype(np.int64)
    return dict(N_s=N_s, R=R, M=M, N=N, N_f=N_f, f_r=f_r, T_short=T_short,
                idx=np.mod(kbar - N // 2, N), dfreq=(f_r - 0.5 / dt) + kbar / T_FFT)


def _cpu_lerp(t0, step, tab, t):
    u = (t - t0) / step
    i = np.clip(np.floor(u), 0, len(tab) - 2).astype(np.int64)
    f = u - i
    return tab[i] + f * (tab[i + 1] - tab[i])


def _cpu_detector(x, det, cfg, pl, a_p, tasc_rel, P):
    """Spectra F_a, F_b [M][N_f] (complex64) and segment norms [3][M] of one detector for
    one circular-orbit template: FP64 timing at knots (Eqs. t-ssb-equation, tau-equation)
    with an FP64 cubic between knots, FP32 windowed-sinc interpolation (2D+1 Hamming taps)
    and heterodyne correction, FP32 weights a/sigma^2, b/sigma^2, and complex64 zero-padded
    FFTs (SciPy pocketfft) of each segment at the output bins."""
    import scipy.fft
    dt, D, N_t = cfg.dt, cfg.D, x.shape[0]
    N_s, M, N, N_f = pl["N_s"], pl["M"], pl["N"], pl["N_f"]
    nsft = int(round(cfg.T_sft / dt))
    n = M * N_s
    # FP64 knots tau_k = (k - 1) CPU_KNOT dt: the binary delay b = R/c at u = tau + b and the
    # SSB delay Delta at t = u - Delta, each by fixed point; d = tau - t = Delta - b
    nk = (n + CPU_KNOT - 1) // CPU_KNOT + 3
    tk = (np.arange(nk, dtype=np.float64) - 1.0) * CPU_KNOT * dt
    bk = np.zeros(nk)
    for _ in range(8):
        bk = a_p * np.sin(2.0 * np.pi * ((tk + bk - tasc_rel) / P))
    dl = _cpu_lerp(det.eph_t0, det.eph_dt, det.ssb_delay, tk + bk)
    for _ in range(8):
        dl = _cpu_lerp(det.eph_t0, det.eph_dt, det.ssb_delay, tk + bk - dl)
    dk = dl - bk
    w = (0.54 - 0.46 * np.cos(2.0 * np.pi * np.arange(2 * D + 1) / (2 * D))).astype(np.float32)
    sig = np.asarray(det.sigma, np.float64)
    pre = np.exp(-2j * np.pi * ((pl["f_r"] * np.arange(N_s) * dt) % 1.0)).astype(np.complex64)
    Fa = np.empty((M, N_f), np.complex64)
    Fb = np.empty((M, N_f), np.complex64)
    norms = np.empty((3, M), np.float32)
    for K0 in range(0, M, CPU_SEG_CHUNK):
        K1 = min(M, K0 + CPU_SEG_CHUNK)
        r = np.arange(K0 * N_s, K1 * N_s, dtype=np.int64)
        k = r // CPU_KNOT
        h = (r - k * CPU_KNOT) / CPU_KNOT
        d = (-h * (h - 1) * (h - 2) / 6.0 * dk[k] + (h + 1) * (h - 1) * (h - 2) / 2.0 * dk[k + 1]
             - (h + 1) * h * (h - 2) / 2.0 * dk[k + 2] + (h + 1) * h * (h - 1) / 6.0 * dk[k + 3])
        g = 0.5 - d / dt                         # t/dt = r - d/dt; j* = round half up
        fl = np.floor(g)
        jstar = r + fl.astype(np.int64)
        delta = ((g - 0.5) - fl).astype(np.float32)
        # windowed sinc with sin(pi (delta - m)) = (-1)^m sin(pi delta)
        sp = (np.sin(np.float32(np.pi) * delta) / np.float32(np.pi)).astype(np.float32)
        zero = delta == 0.0
        acc = np.zeros(r.shape, np.complex64)
        for m in range(-D, D + 1):
            j = jstar + m
            ok = (j >= 0) & (j < N_t)
            xv = np.where(ok, x[np.clip(j, 0, N_t - 1)], np.complex64(0))
            with np.errstate(divide="ignore", invalid="ignore"):
                c = w[m + D] * ((-sp if m & 1 else sp) / (delta - np.float32(m)))
            c = np.where(zero, np.float32(1.0 if m == 0 else 0.0), c).astype(np.float32)
            acc += xv * c
        acc *= np.exp(-2j * np.pi * ((cfg.f_h * d) % 1.0)).astype(np.complex64)
        # weights at the detector time (j* + delta) dt
        tt = (jstar + delta.astype(np.float64)) * dt
        a = _cpu_lerp(det.ab_t0, det.ab_dt, det.a_tab, tt).astype(np.float32)
        b = _cpu_lerp(det.ab_t0, det.ab_dt, det.b_tab, tt).astype(np.float32)
        q = np.floor_divide(jstar, nsft)
        blk = np.where((jstar - q * nsft == 0) & (delta < 0), q - 1, q)
        ok = (blk >= 0) & (blk < len(sig))
        s = np.where(ok, sig[np.clip(blk, 0, len(sig) - 1)], 0.0).astype(np.float32)
        s2 = s * s
        inv = np.where(s > 0, 1.0 / np.where(s > 0, s2, 1.0), 0.0).astype(np.float32)
        al, be = a * inv, b * inv
        nseg = K1 - K0
        norms[0, K0:K1] = (al * al * s2).reshape(nseg, N_s).sum(axis=1)
        norms[1, K0:K1] = (be * be * s2).reshape(nseg, N_s).sum(axis=1)
        norms[2, K0:K1] = (al * be * s2).reshape(nseg, N_s).sum(axis=1)
        ph = np.exp(-2j * np.pi * (np.outer(np.arange(K0, K1) * pl["T_short"], pl["dfreq"]) % 1.0))
        ph = ph.astype(np.complex64)
        for wt, out in ((al, Fa), (be, Fb)):
            y = (acc * wt).reshape(nseg, N_s) * pre
            out[K0:K1] = scipy.fft.fft(y, n=N, axis=1, workers=1)[:, pl["idx"]] * ph
    return Fa, Fb, norms


def _cpu_pairs(F, norms, Q, M, R, mode):
    """Re sum over the pair set of conj(F_a,XK) F_a,YL + conj(F_b,XK) F_b,YL (FP32) and the
    normalisation sum of A_K A_L + B_K B_L + 2 C_K C_L (Eq. final-formatted-rho; each
    unordered pair once unless mode = 2, every ordered pair, or 1, cross-detector only)."""
    N_f = F[0][0].shape[1]
    raw = np.zeros(N_f, np.float32)
    Dn = 0.0
    for X in range(Q):
        for Y in range(Q):
            for lag in range(-R, R + 1):
                if not (mode == 2 or X < Y or (X == Y and mode == 0 and lag >= 1)):
                    continue
                a, b = max(0, -lag), min(M, M - lag)
                if a >= b:
                    continue
                for c in (0, 1):
                    raw += (np.conj(F[X][c][a:b]) * F[Y][c][a + lag:b + lag]).real.sum(axis=0, dtype=np.float32)
                nx, ny = norms[X], norms[Y]
                Dn += float(np.sum(nx[0][a:b] * ny[0][a + lag:b + lag] + nx[1][a:b] * ny[1][a + lag:b + lag]
                                   + 2.0 * nx[2][a:b] * ny[2][a + lag:b + lag], dtype=np.float64))
    return raw, Dn


def cpu_fp32_rho(ds, templates, threads=None):
    """rho [template][bin] by the plain FP32 CPU implementation, templates spread over
    `threads` host threads (default: every core).  Circular orbits."""
    from concurrent.futures import ThreadPoolExecutor
    cfg = ds.cfg
    pl = _cpu_plan(cfg)
    xs = [np.ascontiguousarray(np.asarray(ds.x[q]).astype(np.complex64)) for q in range(len(ds.dets))]
    tm = np.asarray(templates, np.float64)

    def one(row):
        F, nm = [], []
        for q, det in enumerate(ds.dets):
            Fa, Fb, norms = _cpu_detector(xs[q], det, cfg, pl, float(row[0]), float(row[1]) - cfg.t0, float(row[2]))
            F.append((Fa, Fb))
            nm.append(norms)
        raw, Dn = _cpu_pairs(F, nm, len(ds.dets), pl["M"], pl["R"], cfg.pair_mode)
        return (math.sqrt(2.0) * raw / math.sqrt(Dn)).astype(np.float32) if Dn > 0 else np.zeros_like(raw)

    with ThreadPoolExecutor(max_workers=threads or os.cpu_count()) as ex:
        return np.stack(list(ex.map(one, tm)))


def cpu_fp32_baseline(ds, n_templates=16):
    """Time the FP32 CPU implementation on the first n_templates of the workload's grid,
    every core busy (templates are independent, so the rate scales per template)."""
    threads = min(os.cpu_count() or 1, n_templates)
    t = time.perf_counter()
    rho = cpu_fp32_rho(ds, ds.templates[:n_templates], threads)
    sec = time.perf_counter() - t
    return {"value": rho.size / sec, "unit": UNIT, "cores": threads, "kind": "fp32_pocketfft",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"{n_templates} templates x {rho.shape[1]} bins of the full workload ({sec:.1f} s), "
                      f"one template per thread"}


# ---------------------------------------------------------------------------
# GPU run
# ---------------------------------------------------------------------------
def algorithmic_costs(plan_info, Q, n_t, D=8, learned=False):
    """Algorithmic flops / bytes of the path for n_t templates.

    Whole-path flops per template: FFT at 5 N log2 N per zero-padded segment
    transform (2 weights x Q detectors x M segments); per source sample and
    detector, 8 flops per windowed-sinc tap (coefficient and complex multiply-add,
    2D+1 taps) or 4 per learned tap (8 taps, plus 16 for the tap-table
    interpolation), + 30 for timing, phase and weights; pair sum at 8 flops per (detector,
    segment, weight, bin) and partner (2R + 2 partners).  Staged kernels: bytes each
    reads and writes."""
    N = plan_info["N_FFT"]
    M, N_f, N_tau, R = plan_info["M"], plan_info["N_f"], plan_info["N_tau"], plan_info["R"]
    fft = 2 * Q * M * 5.0 * N * math.log2(N)
    per_sample = (4.0 * 8 + 16.0) if learned else 8.0 * (2 * D + 1)
    interp = Q * N_tau * (per_sample + 30.0)
    pairs = 2 * Q * M * N_f * 8.0 * (2 * R + 2)
    return {
        "fft_flops": fft * n_t, "interp_flops": interp * n_t, "pair_flops": pairs * n_t,
        "total_flops": (fft + interp + pairs) * n_t,
        "resample_bytes": n_t * (Q * 2 * N_tau * 8 + Q * M * 16),
        "segfft_bytes": n_t * (Q * 2 * N_tau * 8 + Q * M * 2 * N_f * 8),
        "pair_bytes": n_t * (Q * M * 2 * N_f * 8 + N_f * 4),
    }


def run_gpu(args):
    import torch
    import synth
    import paper_1712_06515_gb300 as cc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    long_lag = args.workload == "o1_long"
    ds = synth.o1_band(seed=1002, T_max=36000.0 if long_lag else 3600.0)
    from paper_1712_06515_gb300 import sharding
    B = args.templates
    grid = ds.templates
    # weak scaling: rank r takes its contiguous block of a global batch of world x B
    # templates (the grid repeated as needed)
    t_start, t_stop = sharding.shard_range(world * B, rank, world)
    idx = np.arange(t_start, t_stop) % grid.shape[0]
    # template rows (a_p, T_asc, P, e, omega): the circular grid with e = omega = 0
    tm_host = np.ascontiguousarray(np.concatenate([grid[idx], np.zeros((B, 2))], axis=1))
    if args.eccentricity:
        tm_host[:, 3], tm_host[:, 4] = args.eccentricity, 0.7
    if args.pair_mode == "all_ordered":
        ds.cfg.pair_mode = 2
    learned = args.interp == "learned"
    plan = cc.CrossCorrPlan(ds.cfg, ds.dets, interp=cc.INTERP_LEARNED if learned else cc.INTERP_EXACT,
                            store=cc.STORE_BF16 if long_lag else cc.STORE_FP32)
    if args.chunk_waves or args.batch_templates:
        plan.set_tuning(batch_templates=args.batch_templates, chunk_waves=args.chunk_waves)
    if args.search_path != "auto":
        plan.set_path({"fused": cc.PATH_FUSED, "two_pass": cc.PATH_TWO_PASS, "staged": cc.PATH_STAGED}[args.search_path])
    Q, N_f = plan.Q, plan.N_f
    path = plan.search_path
    x = torch.from_numpy(ds.x64).to(dev)
    tm = torch.from_numpy(tm_host).to(dev)
    rho = torch.empty((B, N_f), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    lib = cc.load()

    def step():
        plan.search(x, tm, rho)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    plan.kernel_time()            # clear
    plan.set_kernel_timing(True)  # event pair around every dominant-kernel launch, same stream
    n0 = lib.crosscorr_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = lib.crosscorr_kernel_launches() - n0
    plan.set_kernel_timing(False)
    fused_ms, fused_launches = plan.kernel_time()
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1000.0
    if dist:
        t = torch.tensor([elapsed], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
        dist.barrier()
    units = world * B * N_f * args.steps
    value = units / elapsed

    # per-template timing of the staged kernels (same work, events between the launches),
    # reported beside the fused number
    info = plan.info
    nb = min(B, 2)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    tms = tm[:nb]
    for rep in range(2):
        evs[0].record(stream)
        ab, nrm = plan.resample(x, tms)
        evs[1].record(stream)
        F = plan.segment_fft(ab, nb)
        evs[2].record(stream)
        plan.pair_accumulate(F, nrm, nb)
        evs[3].record(stream)
    torch.cuda.synchronize()
    stage_ms = {"resample": evs[0].elapsed_time(evs[1]) / nb,
                "segment_fft": evs[1].elapsed_time(evs[2]) / nb,
                "pair_accumulate": evs[2].elapsed_time(evs[3]) / nb}
    del ab, nrm, F

    # e2e through the public API: pinned host inputs copied in, rho read back, every step
    x_host = torch.from_numpy(ds.x64).pin_memory()
    tm_pin = torch.from_numpy(tm_host).pin_memory()
    rho_host = torch.empty((B, N_f), dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.e2e_steps):
        xd = x_host.to(dev, non_blocking=True)
        td = tm_pin.to(dev, non_blocking=True)
        r = plan.search(xd, td)
        rho_host.copy_(r, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1000.0
    e2e_value = world * B * N_f * args.e2e_steps / e2e_s

    # the one collective: every rank's top-k (global template indices) merged on the host
    k_hits = 16
    local = plan.topk(rho, k_hits)
    hits = np.zeros(len(local), sharding.HIT_DTYPE)
    for f in ("tmpl", "bin", "freq", "rho"):
        hits[f] = local[f]
    merged = sharding.merge_topk(sharding.globalize(hits, t_start), k_hits)
    peaks, peak_kind = load_peaks()
    out = None
    if rank == 0:
        costs = algorithmic_costs(info, Q, 1, ds.cfg.D, learned)
        # The dominant kernel of the step, timed with CUDA events around its own launches
        # on the launching stream: on the two-pass path the segment-spectrum + pair-sum
        # kernel (its algorithmic flops: FFT + pairs; resampling is the other kernel), on
        # the fused path the one-pass kernel (all flops).  Against the FP32-ALU roofline
        # from the SM count, FP32 lanes and the maximum SM clock.
        if path == cc.PATH_TWO_PASS:
            kname, kflops = spectrum_kernel_name(info, long_lag), costs["fft_flops"] + costs["pair_flops"]
        else:
            kname, kflops = "fused_kernel", costs["total_flops"]
        achieved = kflops * B * args.steps / (fused_ms / 1e3) / 1e12
        peak, peak_how = fp32_peak(cc, clk)
        other_ms = max(0.0, 1e3 * elapsed - fused_ms) / (B * args.steps)
        traffic = None
        if path == cc.PATH_TWO_PASS and SEGPAIR_DRAM_BYTES_PER_TEMPLATE is not None and fused_launches \
                and not long_lag and kname == "segpair_tma_kernel" and not learned and args.pair_mode == "unordered":
            traffic = SEGPAIR_DRAM_BYTES_PER_TEMPLATE * B * args.steps / fused_launches
        # the staged stage kernels are HBM-bound: algorithmic bytes (input read once,
        # output written once) over their event-timed duration, against the measured copy peak
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        sbytes = {"resample": costs["resample_bytes"] + Q * ds.cfg.n_samples * 8,
                  "segment_fft": costs["segfft_bytes"], "pair_accumulate": costs["pair_bytes"]}
        staged_hbm = {k: {"GB/s": sbytes[k] / (stage_ms[k] / 1e3) / 1e9,
                          "frac": sbytes[k] / (stage_ms[k] / 1e3) / 1e9 / hbm,
                          "bytes_per_template": sbytes[k]} for k in sbytes}
        staged_hbm["peak_GB/s"] = hbm
        staged_hbm["peak_kind"] = f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu capture, scaled by templates per launch)",
                "peak_kind": peak_how,
                "flops_per_template": kflops,
                "kernel_ms_per_launch": fused_ms / max(fused_launches, 1),
                "kernel_launches": fused_launches, "kernel_share_of_step": fused_ms / (1e3 * elapsed),
                "other_kernels_ms_per_template": other_ms,
                "staged_ms_per_template": stage_ms, "staged_hbm": staged_hbm}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": ("o1_long: 2 det, 120 d at 60% duty, 0.5 Hz at 150 Hz, T_sft=360 s, "
                                    "T_max=T_short=36000 s, BF16 storage of the resampled series, "
                                    "40x200 orbital grid") if long_lag else
                                   ("o1_band: 2 det, 120 d at 60% duty, 0.5 Hz at 150 Hz, "
                                    "T_sft=360 s, T_max=T_short=3600 s, 40x200 orbital grid"),
                       "templates_per_step_per_rank": B, "grid_templates": GRID_TEMPLATES,
                       "N_f": N_f, "N_FFT": info["N_FFT"], "M": info["M"], "L": info["L"], "C": info["C"],
                       "l2": "inputs larger than L2 (2 x 83 MB complex64 series)",
                       "timing_precision": "f64 knots, f32 interpolation/FFT/pairs"
                                           + (", bf16 storage of a_r, b_r" if long_lag else ""),
                       "search_path": {cc.PATH_FUSED: "fused (one cluster kernel)",
                                       cc.PATH_TWO_PASS: "two-pass (resample to HBM, then spectra + pairs)",
                                       cc.PATH_STAGED: "staged"}[path],
                       "interp": ("learned 8-tap network (bf16 weights, tabulated taps)" if learned
                                  else f"windowed sinc, {2 * ds.cfg.D + 1} taps"),
                       "pair_mode": args.pair_mode,
                       "eccentricity": args.eccentricity},
            "roofline": roof,
            "clocks": clk,
            "topk": {"k": k_hits, "merged_from_ranks": world,
                     "best": {"template": int(merged["tmpl"][0]), "grid_template": int(merged["tmpl"][0]) % grid.shape[0],
                              "bin": int(merged["bin"][0]), "freq": float(merged["freq"][0]),
                              "rho": float(merged["rho"][0])}},
            "gpu_launches": int(launches),
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(x_host.numel() * 8 + tm_pin.numel() * 8),
                    "d2h_bytes_per_step": int(rho_host.numel() * 4)},
        }
        if world == 1 and not args.no_variants and args.workload == "o1_band":
            out["variants"] = run_variants(args, ds, x, tm_host, plan, peak)
        if world == 1 and not args.no_cpu_baseline and args.workload == "o1_band" and not learned \
                and args.eccentricity == 0.0:
            out["cpu_fp32_baseline"] = cpu_fp32_baseline(ds)
        if world == 1 and not args.no_cpu_baseline:
            v, dt, n = cpu_oracle_baseline(args.cpu_days)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                                   "sample": f"1 template x {N_f} bins over the first {args.cpu_days:g} "
                                             f"of 120 days, {n} runs ({dt:.1f} s), scaled linearly to 120 d"}
        print(json.dumps(out), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


def _time_search(plan, x, tm, steps, warmup=1):
    """ms per search of `tm` (CUDA events on the current stream) and the spectrum kernel's
    share, after `warmup` untimed searches."""
    import torch
    stream = torch.cuda.current_stream()
    rho = torch.empty((tm.shape[0], plan.N_f), dtype=torch.float32, device=x.device)
    for _ in range(warmup):
        plan.search(x, tm, rho)
    plan.kernel_time()
    plan.set_kernel_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.search(x, tm, rho)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.set_kernel_timing(False)
    kms, _ = plan.kernel_time()
    plan.check()
    return e0.elapsed_time(e1) / steps, kms / steps, rho


def variant_stencils(args, ds, x, tm_host, plan, peak):
    """Learned 8-tap interpolation against the exact 17-tap windowed sinc on the 120-day
    band: speed on the first 512 templates of the grid, and accuracy on a noiseless
    injection against the widest exact stencil (D = 32, 65 taps) as the judge."""
    import torch
    import synth
    import paper_1712_06515_gb300 as cc
    dev = x.device
    B = min(512, tm_host.shape[0])
    tm = torch.from_numpy(np.ascontiguousarray(tm_host[:B])).to(dev)
    res = {"templates": B}
    with cc.CrossCorrPlan(ds.cfg, ds.dets, interp=cc.INTERP_LEARNED) as lp:
        for name, pl, learned in (("exact_d8", plan, False), ("learned", lp, True)):
            ms, kms, _ = _time_search(pl, x, tm, steps=2)
            kfl = algorithmic_costs(pl.info, pl.Q, 1, ds.cfg.D, learned)
            res[name] = {"value": B * pl.N_f / (ms / 1e3), "unit": UNIT, "ms_per_template": ms / B,
                         "other_kernels_ms_per_template": (ms - kms) / B,
                         "spectrum_frac": (kfl["fft_flops"] + kfl["pair_flops"]) * B / (kms / 1e3) / 1e12 / peak}
    # accuracy: noiseless injection, the injected template and three grid neighbours
    dn = synth.o1_band(seed=1002, noise=False)
    inj = dn.injection
    ap = np.linspace(1.36, 1.52, 40)
    ta = inj.T_asc + np.linspace(-300.0, 300.0, 200)
    pick = np.array([[inj.a_p, inj.T_asc, inj.P], [ap[19], ta[99], inj.P], [ap[20], ta[101], inj.P],
                     [ap[21], ta[100], inj.P]])
    tmi = torch.from_numpy(np.ascontiguousarray(np.concatenate([pick, np.zeros((4, 2))], axis=1))).to(dev)
    xn = torch.from_numpy(dn.x64).to(dev)
    out = {}
    for name, D, interp in (("judge_exact_d32", 32, cc.INTERP_EXACT), ("exact_d8", 8, cc.INTERP_EXACT),
                            ("learned", 8, cc.INTERP_LEARNED)):
        cfg = dataclass_replace(dn.cfg, D=D)
        with cc.CrossCorrPlan(cfg, dn.dets, interp=interp) as pl:
            out[name] = pl.search(xn, tmi).cpu().numpy().astype(np.float64)
            pl.check()
    judge = out["judge_exact_d32"]
    peak_rho = float(np.abs(judge).max())
    for name in ("exact_d8", "learned"):
        err = np.abs(out[name] - judge).max(axis=1)
        res[name]["rho_err_vs_judge"] = float(err.max())
        res[name]["rel_err_vs_judge"] = float(err.max() / peak_rho)
        res[name]["argmax_equal"] = bool(np.unravel_index(np.argmax(out[name]), judge.shape)
                                         == np.unravel_index(np.argmax(judge), judge.shape))
    res["judge"] = "exact windowed sinc D = 32 (65 taps), noiseless injection, max rho %.2f" % peak_rho
    res["learned_faster"] = res["learned"]["value"] > res["exact_d8"]["value"]
    res["learned_at_least_as_accurate"] = res["learned"]["rho_err_vs_judge"] <= res["exact_d8"]["rho_err_vs_judge"]
    return res


def variant_long_lag(args, peak):
    """The long-lag precision variant: T_max = T_short = 36000 s (N_FFT = 2^18, 123564
    bins) with BF16 storage of the resampled series, 64 templates of the grid; rho error
    of BF16 storage against FP32 storage (the FP32 path's own oracle parity is 1e-4)."""
    import torch
    import synth
    import paper_1712_06515_gb300 as cc
    dev = torch.device("cuda", torch.cuda.current_device())
    dl = synth.o1_band(seed=1002, T_max=36000.0)
    B = 64
    tm = torch.from_numpy(np.ascontiguousarray(np.concatenate([dl.templates[:B], np.zeros((B, 2))], axis=1))).to(dev)
    x = torch.from_numpy(dl.x64).to(dev)
    res = {"templates": B}
    with cc.CrossCorrPlan(dl.cfg, dl.dets, store=cc.STORE_BF16) as pl:
        ms, kms, _ = _time_search(pl, x, tm, steps=2)
        kfl = algorithmic_costs(pl.info, pl.Q, 1, dl.cfg.D, False)
        res.update({"value": B * pl.N_f / (ms / 1e3), "unit": UNIT, "ms_per_template": ms / B,
                    "kernel": spectrum_kernel_name(pl.info, True),
                    "spectrum_frac": (kfl["fft_flops"] + kfl["pair_flops"]) * B / (kms / 1e3) / 1e12 / peak,
                    "spectrum_share": kms / ms, "N_f": pl.N_f, "N_FFT": pl.info["N_FFT"]})
        inj = dl.injection
        two = torch.from_numpy(np.array([[inj.a_p, inj.T_asc, inj.P, 0.0, 0.0],
                                         [1.52, inj.T_asc + 300.0, inj.P, 0.0, 0.0]])).to(dev)
        bf = pl.search(x, two).cpu().numpy().astype(np.float64)
        pl.check()
    with cc.CrossCorrPlan(dl.cfg, dl.dets, store=cc.STORE_FP32) as pf:
        f32 = pf.search(x, two).cpu().numpy().astype(np.float64)
        pf.check()
    err = np.abs(bf - f32).max(axis=1)
    lim = np.maximum(1.0, np.abs(f32).max(axis=1))
    res["rho_err_bf16_vs_fp32"] = [float(e) for e in err]
    res["rel_err_bf16_vs_fp32"] = [float(e) for e in err / lim]
    return res


def variant_multiband(args, peak, scale=0.05):
    """The batched multi-band workload at a reduced template scale: one CUDA graph launch
    per step over 32 bands after per-band autotuning."""
    import torch
    import synth
    import paper_1712_06515_gb300 as cc
    from paper_1712_06515_gb300.multiband import MultiBandSearch
    dev = torch.device("cuda", torch.cuda.current_device())
    datasets = synth.multiband(template_scale=scale)
    bands = [(d.cfg, d.dets, torch.from_numpy(d.x64).to(dev), torch.from_numpy(d.templates).to(dev))
             for d in datasets]
    mb = MultiBandSearch(bands, tune=True, tune_templates=32).capture()
    stream = torch.cuda.current_stream()
    mb.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(2):
        mb.run()
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1000.0 / 2
    flops = sum(algorithmic_costs(p.info, p.Q, tm.shape[0], cfg.D, False)["total_flops"]
                for p, (cfg, _, _, tm) in zip(mb.plans, bands))
    res = {"template_scale": scale, "templates": int(sum(t.shape[0] for (_, _, _, t) in bands)),
           "value": mb.units / sec, "unit": UNIT, "ms_per_step": 1e3 * sec,
           "graph_frac": flops / sec / 1e12 / peak, "kernels_per_step": mb.kernels_per_run}
    mb.close()
    return res


def run_variants(args, ds, x, tm_host, plan, peak):
    """Variants measured after the headline in the same process and under one clock
    sampler (rank 0, one GPU): learned vs exact stencil, long-lag BF16, multi-band."""
    import torch
    res = {}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for name, fn in (("stencils", lambda: variant_stencils(args, ds, x, tm_host, plan, peak)),
                     ("long_lag_bf16", lambda: variant_long_lag(args, peak)),
                     ("multiband", lambda: variant_multiband(args, peak))):
        t0 = time.perf_counter()
        try:
            res[name] = fn()
        except Exception as e:   # noqa: BLE001 - a failed variant is reported, the headline stands
            res[name] = {"error": f"{type(e).__name__}: {e}"}
        res[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()
    res["clocks"] = clocks.stop()
    return res


def dataclass_replace(cfg, **kw):
    import dataclasses
    return dataclasses.replace(cfg, **kw)


def run_multiband(args):
    """32 bands (T_max 240-3600 s, 10 d at 60 % duty), every band's search recorded in one
    CUDA graph after per-band autotuning; a step is one graph launch."""
    import torch
    import synth
    import paper_1712_06515_gb300 as cc
    from paper_1712_06515_gb300.multiband import MultiBandSearch

    dev = torch.device("cuda", 0)
    learned = args.interp == "learned"
    datasets = synth.multiband(template_scale=args.template_scale)
    bands = [(ds.cfg, ds.dets, torch.from_numpy(ds.x64).to(dev), torch.from_numpy(ds.templates).to(dev))
             for ds in datasets]
    mb = MultiBandSearch(bands, interp=cc.INTERP_LEARNED if learned else cc.INTERP_EXACT,
                         tune=True, tune_templates=64).capture()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        mb.run()
    torch.cuda.synchronize()
    lib = cc.load()
    clocks = ClockSampler(0)
    clocks.start()
    n0 = lib.crosscorr_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        mb.run()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = e0.elapsed_time(e1) / 1000.0
    units = mb.units
    value = units * args.steps / elapsed
    # algorithmic flops of the whole graph (every kernel), over the graph's time
    flops = 0.0
    for p, (cfg, dets, x, tm) in zip(mb.plans, bands):
        c = algorithmic_costs(p.info, p.Q, tm.shape[0], cfg.D, learned)
        flops += c["total_flops"]
    achieved = flops * args.steps / elapsed / 1e12
    peak, peak_kind = fp32_peak(cc, clk)
    # e2e: every band's series and templates copied in from pinned memory, rho copied out
    x_host = [x.cpu().pin_memory() for (_, _, x, _) in bands]
    t_host = [t.cpu().pin_memory() for (_, _, _, t) in bands]
    r_host = [torch.empty(r.shape, dtype=r.dtype).pin_memory() for r in mb.rho]
    torch.cuda.synchronize()
    e0.record(stream)
    for (_, _, x, t), xh, th in zip(bands, x_host, t_host):
        x.copy_(xh, non_blocking=True)
        t.copy_(th, non_blocking=True)
    mb.run()
    for r, rh in zip(mb.rho, r_host):
        rh.copy_(r, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e = units / (e0.elapsed_time(e1) / 1000.0)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "multiband: 32 bands of 0.5 Hz over 20-250 Hz, T_sft=T_short=T_max "
                               "240-3600 s, 10 d at 60% duty, one CUDA graph launch per step",
                   "templates_per_step": int(sum(t.shape[0] for (_, _, _, t) in bands)),
                   "template_scale": args.template_scale,
                   "paths": [{1: "fused", 2: "two-pass"}[t["path"]] + (f"/L{t['transform_len']}" if t.get("transform_len") else "")
                             + f"/w{t['chunk_waves']}" for t in mb.tuning],
                   # per band, from the autotuner's timing of its first 64 templates: coset
                   # length, ms per template, fraction of the FP32 peak (algorithmic flops)
                   "bands": [{"L": int(pl.info["L"]), "ms_per_template": round(t["ms"] / min(64, tt.shape[0]), 4),
                              "frac": round(algorithmic_costs(pl.info, pl.Q, 1, cf.D, learned)["total_flops"]
                                            / (t["ms"] / min(64, tt.shape[0]) * 1e-3) / (peak * 1e12), 3)}
                             for pl, t, tt, (cf, _, _, _) in zip(mb.plans, mb.tuning, mb.templates, bands)],
                   "interp": "learned 8-tap" if learned else "windowed sinc, 17 taps",
                   "l2": "inputs: 32 bands x 2 x 6.9 MB series (442 MB, larger than L2)"},
        "roofline": {"bound": "alu", "kernel": "graph (all kernels of all bands)", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                     "peak_kind": peak_kind},
        "clocks": clk,
        # graph replays launch the kernels recorded at capture
        "gpu_launches": int(lib.crosscorr_kernel_launches() - n0) + mb.kernels_per_run * args.steps,
        "e2e": {"value": e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(x.numel() * 8 + t.numel() * 8 for x, t in zip(x_host, t_host))),
                "d2h_bytes_per_step": int(sum(r.numel() * 4 for r in r_host))},
    }
    print(json.dumps(out), flush=True)
    mb.close()


def run_demod(args):
    """The detector-frame (demodulation) statistic on the o1_band workload: SFTs once, then
    a step = crosscorr_demod_search over the template batch (the pair loop of the method, or
    with --demod-form separable the same rho from running window sums)."""
    import torch
    import synth
    import paper_1712_06515_gb300 as cc
    dev = torch.device("cuda", 0)
    long_lag = args.workload == "o1_long"
    ds = synth.o1_band(seed=1002, T_max=36000.0 if long_lag else 3600.0)
    B = args.templates
    tm = cc.templates5(torch.from_numpy(np.ascontiguousarray(ds.templates[:B])).to(dev))
    plan = cc.CrossCorrPlan(ds.cfg, ds.dets)
    x = torch.from_numpy(ds.x64).to(dev)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.demod_prepare(x)
    e1.record(stream)
    torch.cuda.synchronize()
    sft_ms = e0.elapsed_time(e1)
    separable = args.demod_form == "separable"
    plan.set_demod_form(separable)
    rho = torch.empty((B, plan.N_f), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        plan.demod_search(tm, rho)
    torch.cuda.synchronize()
    lib = cc.load()
    n0 = lib.crosscorr_kernel_launches()
    clocks = ClockSampler(0)
    clocks.start()
    plan.kernel_time()            # clear
    plan.set_kernel_timing(True)  # event pair around every pair-loop launch, same stream
    e0.record(stream)
    for _ in range(args.steps):
        plan.demod_search(tm, rho)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    plan.set_kernel_timing(False)
    pair_ms, pair_launches = plan.kernel_time()
    elapsed = e0.elapsed_time(e1) / 1000.0
    units = B * plan.N_f * args.steps
    nsft = int(round(ds.cfg.T_sft / ds.cfg.dt))
    n_blk = ds.cfg.n_samples // nsft
    lk = [np.asarray(d.sigma[:n_blk]) > 0 for d in ds.dets]
    locked = sum(int(np.sum(v)) for v in lk)
    # unordered pairs of distinct SFTs within T_max (every detector pair, lags 0..Rs blocks)
    Rs = int(math.floor(ds.cfg.T_max / ds.cfg.T_sft + 1e-9))
    pairs = 0
    for X in range(len(lk)):
        for Y in range(X, len(lk)):
            for lag in range(0, Rs + 1):
                if X == Y and lag == 0:
                    continue
                a, b = lk[X][: n_blk - lag], lk[Y][lag:]
                pairs += int(np.sum(a & b))
                if X != Y and lag > 0:
                    pairs += int(np.sum(lk[Y][: n_blk - lag] & lk[X][lag:]))
    # algorithmic flops per (template, bin): 12 per pair (the filter weight, Re of the
    # product, the normalisation term, two accumulations) and 30 per locked SFT (two
    # sinc-weighted bins, the phase and its rotation, Xi^2)
    flops_tb = 12.0 * pairs + 30.0 * locked
    if separable:
        # the same 30 per locked SFT for its bin, plus 53 for the factored pair and
        # normalisation terms and the running sums of its block, and 14 per SFT for the
        # window update (28 per block of two detectors): no per-pair term
        flops_tb = (30.0 + 53.0 + 14.0) * locked
    peak, peak_kind = fp32_peak(cc, clk)
    achieved = flops_tb * units / (pair_ms / 1e3) / 1e12 if pair_ms > 0 else None
    out = {
        "metric": METRIC, "value": units / elapsed, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "o1_band: 2 det, 120 d at 60% duty, 0.5 Hz at 150 Hz, T_sft=360 s SFTs, "
                               f"T_max={ds.cfg.T_max:g} s", "method": "detector-frame (demodulation) CrossCorr, n_bin=2",
                   "demod_form": args.demod_form, "templates_per_step": B, "locked_sfts": locked, "sft_pairs": pairs, "sft_ms_once": sft_ms},
        "roofline": {"bound": "alu", "kernel": "demod_sep_kernel" if separable else "demod_pair_kernel",
                     "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak if achieved else None, "traffic": None,
                     "peak_kind": peak_kind, "flops_per_template_bin": flops_tb, "kernel_ms_per_launch": pair_ms / max(1, pair_launches),
                     "kernel_launches": pair_launches,
                     "kernel_share_of_step": pair_ms / (1e3 * elapsed) if elapsed > 0 else None},
        "clocks": clk, "gpu_launches": int(lib.crosscorr_kernel_launches() - n0),
    }
    print(json.dumps(out), flush=True)
    plan.close()


def run_sft_series(args):
    """Appendix B's input preparation at the 120-day band's shape: the locked SFTs of one
    detector (360 bins of a 360 s SFT at 1 s, 60 % of 28800 blocks) to the heterodyned
    series.  Synthetic bins."""
    import torch
    import synth
    import paper_1712_06515_gb300 as cc
    dev = torch.device("cuda", 0)
    ds = synth.o1_band(seed=1002)
    nsft = int(round(ds.cfg.T_sft / ds.cfg.dt))
    n_blocks = ds.cfg.n_samples // nsft
    locked = np.asarray(ds.dets[0].sigma[:n_blocks]) > 0
    block_sft = np.full(n_blocks, -1, np.int64)
    block_sft[locked] = np.arange(int(locked.sum()))
    rng = np.random.default_rng(1002)
    band = torch.from_numpy((rng.standard_normal((int(locked.sum()), nsft))
                             + 1j * rng.standard_normal((int(locked.sum()), nsft))).astype(np.complex64)).to(dev)
    bsd = torch.from_numpy(block_sft).to(dev)
    x = torch.empty(n_blocks * nsft, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        cc.sfts_to_series(band, bsd, ds.cfg.T_sft, ds.cfg.f_h, out=x)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the API calls one after another (host overhead included where it exceeds the kernel)
    e0.record(stream)
    for _ in range(args.steps):
        cc.sfts_to_series(band, bsd, ds.cfg.T_sft, ds.cfg.f_h, out=x)
    e1.record(stream)
    torch.cuda.synchronize()
    api_ms = e0.elapsed_time(e1) / args.steps
    # the same calls captured in a CUDA graph: the kernels back to back, the figure the
    # roofline takes
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(args.steps):
            cc.sfts_to_series(band, bsd, ds.cfg.T_sft, ds.cfg.f_h, out=x)
    graph.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    nbytes = band.numel() * 8 + n_blocks * nsft * 8 + n_blocks * 8
    hbm = float(load_peaks()[0].get("hbm_gbs", 6800.0))
    # N' = 360 = 4 x 2 x 3 x 3 x 5 takes the mixed-radix FFT: 5 N' log2 N' flops per SFT,
    # far below the bytes it moves, so the bound is HBM (read the bands, write the series)
    n_lk = int(locked.sum())
    alg_flops = n_lk * 5.0 * nsft * math.log2(nsft)
    fp32_pk, _ = fp32_peak(cc, clk)
    out = {"metric": "SFT-to-series output samples per second", "value": n_blocks * nsft / (ms / 1e3),
           "unit": "samples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "120 d at 1 s, T_sft = 360 s, one detector", "blocks": n_blocks,
                      "locked_sfts": int(locked.sum()), "bins_per_sft": nsft,
                      "timing": "CUDA graph of the steps' calls; api_ms_per_call: the same calls eager"},
           "api_ms_per_call": api_ms,
           "roofline": {"bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": nbytes / (ms / 1e3) / 1e9 / hbm, "traffic": None, "algorithmic_bytes": nbytes,
                        "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs)",
                        "fft_tflops": alg_flops / (ms / 1e3) / 1e12,
                        "fft_frac_of_fp32_peak": alg_flops / (ms / 1e3) / 1e12 / fp32_pk},
           "clocks": clk, "gpu_launches": args.steps}
    print(json.dumps(out), flush=True)


def run_dft_gemm(args):
    """The tensor-core question for short segments, by measurement: a batched DFT-as-GEMM
    (cuBLAS BF16 through torch.matmul, FP32 accumulation) of the exact shape the direct
    DFT of a segment at the output bins needs -- the real form [2 N_f x 2 N_s] times
    [2 N_s x (segments x detectors x weights x templates)] -- against the library's own
    spectrum + pair-sum kernel on the same band, per template.  The GEMM alone covers only
    the spectra (no pair sums, no resampling) and is single-pass BF16 (the 1e-2 bar; the
    FP32 bar would need a split into several passes)."""
    import torch
    import synth
    import paper_1712_06515_gb300 as cc
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    rows = []
    for b in (0, 2, 6):   # the shortest-segment bands: coset lengths 256 and 512
        ds = synth.multiband_band(b, template_scale=0.25, max_templates=64)
        n_t = ds.templates.shape[0]
        with cc.CrossCorrPlan(ds.cfg, ds.dets) as plan:
            info = plan.info
            x = torch.from_numpy(ds.x64).to(dev)
            tm = torch.from_numpy(ds.templates).to(dev)
            ms, kms, _ = _time_search(plan, x, tm, steps=3)
        N_s, N_f, M, Q = info["N_s"], info["N_f"], info["M"], plan.Q
        cols = M * Q * 2 * n_t
        A = torch.randn(2 * N_f, 2 * N_s, device=dev, dtype=torch.bfloat16)
        B = torch.randn(2 * N_s, cols, device=dev, dtype=torch.bfloat16)
        for _ in range(3):
            torch.mm(A, B)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = 5
        for _ in range(reps):
            C = torch.mm(A, B)
        e1.record(stream)
        torch.cuda.synchronize()
        gms = e0.elapsed_time(e1) / reps
        flops = 2.0 * (2 * N_f) * (2 * N_s) * cols
        rows.append({"band": b, "L": info["L"], "N_s": N_s, "N_f": N_f, "N_FFT": info["N_FFT"], "templates": n_t,
                     "library_spectrum_pair_ms_per_template": kms / n_t, "library_search_ms_per_template": ms / n_t,
                     "dft_gemm_bf16_ms_per_template": gms / n_t, "dft_gemm_tflops": flops / (gms / 1e3) / 1e12,
                     "gemm_flops_over_fft_flops": (4.0 * N_f * N_s) / (5.0 * info["N_FFT"] * math.log2(info["N_FFT"]))})
        del A, B, C
    print(json.dumps({"metric": "DFT-as-GEMM vs FFT spectrum kernel, ms per template", "data": "synthetic",
                      "peaks": load_peaks()[0], "bands": rows}), flush=True)


def launch_ranks(argv, n):
    """`--gpus N` with N > 1 outside a launcher: run this script again under
    torch.distributed.run with N ranks on this node (one per GPU, rendezvous on 127.0.0.1)
    and return its exit status."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *argv]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(sys.argv[1:], args.gpus))
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "multiband":
        run_multiband(args)
        return
    if args.method == "demod":
        run_demod(args)
        return
    if args.method == "sft_series":
        run_sft_series(args)
        return
    if args.method == "dft_gemm":
        run_dft_gemm(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
