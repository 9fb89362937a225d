"""GB300 resampled cross-correlation (CrossCorr) search: Python binding.

A thin marshalling layer over the C ABI of ``include/crosscorr.h``: every step
of the statistic (timing, resampling, weighting, segment FFTs, pair sums,
normalisation, top-k) runs in the CUDA library.  PyTorch supplies device
memory and streams only.  Calls fail loudly when the compiled library is
missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, byref, c_double, c_int64, c_void_p
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import CcConfig, CcDetector, CcHit, CcLearnedInterp, CcPlanInfo, CcTuning, CrossCorrError, check

__all__ = ["CrossCorrPlan", "CrossCorrError", "sfts_to_series", "metric", "lattice", "templates5", "PAIR_UNORDERED", "PAIR_CROSS_ONLY",
           "PAIR_ALL_ORDERED", "STORE_FP32", "STORE_BF16", "build", "load"]

PAIR_UNORDERED, PAIR_CROSS_ONLY, PAIR_ALL_ORDERED = 0, 1, 2
STORE_FP32, STORE_BF16 = 0, 1
INTERP_EXACT, INTERP_LEARNED = 0, 1
PATH_AUTO, PATH_FUSED, PATH_TWO_PASS, PATH_STAGED = 0, 1, 2, 3

build = _lib.build
load = _lib.load


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dptr(t) -> int:
    return int(t.data_ptr())


def _check_tensor(name, t, dtype, device_required=True):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if device_required and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def templates5(templates):
    """Template rows as the C ABI's cc_template (a_p, T_asc, P, e, omega): [n, 3]
    circular rows get e = omega = 0; [n, 5] rows are returned as they are."""
    import torch
    if templates.shape[-1] == 5:
        return templates
    z = torch.zeros((templates.shape[0], 2), dtype=templates.dtype, device=templates.device)
    return torch.cat([templates, z], dim=1).contiguous()


def metric(T_obs: float, T_sft: float, T_max: float, Q: int, f: float, a_p: float, T_asc: float, P: float,
           t0: float = 0.0) -> np.ndarray:
    """Phase-mismatch metric g [3, 3] for (a_p, T_asc, P) of a circular orbit (host, in the
    library)."""
    lib = _lib.load()
    orb = np.array([a_p, T_asc, P, 0.0, 0.0], np.float64)
    g = np.zeros(9, np.float64)
    check("crosscorr_metric", lib.crosscorr_metric(float(T_obs), float(T_sft), float(T_max), int(Q), float(f),
                                                   orb.ctypes.data_as(c_void_p), float(t0),
                                                   g.ctypes.data_as(POINTER(c_double))))
    return g.reshape(3, 3)


def lattice(g, mu: float, lo, hi) -> np.ndarray:
    """Cubic template lattice [n, 3] (a_p, T_asc, P) with spacing sqrt(mu / g_ii) over
    [lo, hi] (host, in the library)."""
    lib = _lib.load()
    g = np.ascontiguousarray(g, np.float64).ravel()
    lo = np.ascontiguousarray(lo, np.float64)
    hi = np.ascontiguousarray(hi, np.float64)
    n = c_int64()
    P = POINTER(c_double)
    args = (g.ctypes.data_as(P), float(mu), lo.ctypes.data_as(P), hi.ctypes.data_as(P))
    check("crosscorr_lattice", lib.crosscorr_lattice(*args, None, 0, byref(n)))
    out = np.zeros((n.value, 5), np.float64)
    check("crosscorr_lattice", lib.crosscorr_lattice(*args, out.ctypes.data_as(c_void_p), n.value, byref(n)))
    return out[:, :3].copy()


def measure_fp32_peak(stream=None) -> float:
    """Measured FP32 FMA throughput of the current device in TFLOP/s (diagnostic)."""
    lib = load()
    v = c_double()
    check("crosscorr_measure_fp32_peak", lib.crosscorr_measure_fp32_peak(byref(v), _stream_handle(stream)))
    return v.value


def sfts_to_series(band, block_sft, T_sft: float, f_h: float, out=None, stream=None):
    """Heterodyned, downsampled series [n_blocks * N'] (CUDA complex64) from SFT bands
    band [n_sft, N'] (CUDA complex64) and block_sft [n_blocks] (CUDA int64, -1 = gap):
    the input preparation of Appendix B, in the CUDA library.  ``out``: an optional
    preallocated contiguous complex64 tensor of n_blocks * N' elements."""
    import torch
    lib = _lib.load()
    _check_tensor("band", band, torch.complex64)
    _check_tensor("block_sft", block_sft, torch.int64)
    if band.dim() != 2:
        raise ValueError("band must be [n_sft, N']")
    n_blocks, n_prime = block_sft.numel(), band.shape[1]
    if band.shape[0] == 0:      # every block a gap: the library still takes a valid band pointer
        band = torch.zeros((1, n_prime), dtype=torch.complex64, device=band.device)
    if out is None:
        x = torch.empty(n_blocks * n_prime, dtype=torch.complex64, device=band.device)
    else:
        _check_tensor("out", out, torch.complex64)
        if out.numel() != n_blocks * n_prime:
            raise ValueError("out must hold n_blocks * N' elements")
        x = out
    check("crosscorr_sfts_to_series", lib.crosscorr_sfts_to_series(
        _dptr(band), _dptr(block_sft), n_blocks, n_prime, float(T_sft), float(f_h), _dptr(x),
        _stream_handle(stream)))
    return x


class CrossCorrPlan:
    """A plan for one band: derived FFT/bin layout plus device copies of the tables.

    ``cfg`` needs the attributes t0, dt, n_samples, f_h, f_band, T_sft, T_max,
    T_short, mu_f, D, n_det, pair_mode; each detector in ``dets`` needs eph_t0,
    eph_dt, ssb_delay, ab_t0, ab_dt, a_tab, b_tab, sigma (numpy arrays for the
    tables; times relative to t0).  With ``interp=INTERP_LEARNED`` the learned
    8-tap interpolator is installed from ``learned_weights`` (a weight file; the
    packaged one by default) at the band half-width ``nu_c`` (by default the one
    ``learned_interp.band_halfwidth`` gives for this band).
    """

    def __init__(self, cfg, dets: Sequence, store: int = STORE_FP32, interp: int = INTERP_EXACT,
                 pair_mode: Optional[int] = None, learned_weights: Optional[str] = None,
                 nu_c: Optional[float] = None):
        self._lib = _lib.load()
        c = CcConfig()
        c.t0, c.dt, c.f_h, c.f_band = cfg.t0, cfg.dt, cfg.f_h, cfg.f_band
        c.T_sft, c.T_short, c.T_max, c.mu_f = cfg.T_sft, cfg.T_short, cfg.T_max, cfg.mu_f
        c.n_det, c.D, c.interp, c.store = len(dets), cfg.D, interp, store
        c.pair_mode = cfg.pair_mode if pair_mode is None else pair_mode
        c.n_samples = cfg.n_samples
        self.cfg = c
        keep = []
        arr = (CcDetector * len(dets))()
        for i, d in enumerate(dets):
            ssb = np.ascontiguousarray(d.ssb_delay, np.float64)
            a = np.ascontiguousarray(d.a_tab, np.float64)
            b = np.ascontiguousarray(d.b_tab, np.float64)
            s = np.ascontiguousarray(d.sigma, np.float64)
            keep += [ssb, a, b, s]
            arr[i].ssb_delay = ssb.ctypes.data_as(POINTER(c_double))
            arr[i].eph_t0, arr[i].eph_dt, arr[i].n_eph = d.eph_t0, d.eph_dt, ssb.size
            arr[i].a_tab = a.ctypes.data_as(POINTER(c_double))
            arr[i].b_tab = b.ctypes.data_as(POINTER(c_double))
            arr[i].ab_t0, arr[i].ab_dt, arr[i].n_ab = d.ab_t0, d.ab_dt, a.size
            arr[i].sigma = s.ctypes.data_as(POINTER(c_double))
            arr[i].n_sigma = s.size
        h = c_void_p()
        check("crosscorr_plan", self._lib.crosscorr_plan(byref(c), arr, byref(h)))
        self._h = h
        info = CcPlanInfo()
        self.freqs = np.empty(0)
        check("crosscorr_plan_info", self._lib.crosscorr_plan_info(h, byref(info), None, None))
        self.freqs = np.empty(info.N_f, np.float64)
        self.kbar = np.empty(info.N_f, np.int64)
        check("crosscorr_plan_info", self._lib.crosscorr_plan_info(
            h, byref(info), self.freqs.ctypes.data_as(POINTER(c_double)),
            self.kbar.ctypes.data_as(POINTER(c_int64))))
        self.info = {name: getattr(info, name) for name, _ in CcPlanInfo._fields_}
        self.Q = len(dets)
        self.N_f = info.N_f
        self.M = info.M
        self.N_tau = info.N_tau
        self.store = store
        self.interp = interp
        self.nu_c = None
        if interp == INTERP_LEARNED:
            self.set_learned_interp(learned_weights, nu_c)

    def set_learned_interp(self, path: Optional[str] = None, nu_c: Optional[float] = None):
        """Install (or replace) the learned interpolator's weights; tabulates its taps."""
        from . import learned_interp
        z = np.load(path or learned_interp.WEIGHTS)
        layers = [np.asarray(z[k], np.float32) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
        bits = np.ascontiguousarray(learned_interp.flat_bf16_bits(layers))
        lo, hi = (float(v) for v in z["nu_c_range"])
        if int(z["tap_offset"]) != 3 or str(z["activation"]) != "tanh":
            raise ValueError("the library evaluates tanh networks with taps from floor(t) - 3")
        if nu_c is None:
            nu_c = learned_interp.band_halfwidth(self.cfg.f_band, self.cfg.f_h, self.cfg.dt)
        li = CcLearnedInterp()
        li.weights_bf16 = bits.ctypes.data_as(POINTER(ctypes.c_uint16))
        li.n_weights = bits.size
        li.nu_lo, li.nu_hi, li.nu_c = lo, hi, float(nu_c)
        check("crosscorr_plan_set_learned_interp",
              self._lib.crosscorr_plan_set_learned_interp(self._h, byref(li)))
        self.nu_c = float(nu_c)

    # -- helpers ---------------------------------------------------------------
    def _xptrs(self, x):
        import torch
        if isinstance(x, torch.Tensor):
            xs = [x[i] for i in range(x.shape[0])]
        else:
            xs = list(x)
        if len(xs) != self.Q:
            raise ValueError(f"need {self.Q} detector series, got {len(xs)}")
        for i, xi in enumerate(xs):
            _check_tensor(f"x[{i}]", xi, torch.complex64)
            if xi.numel() != self.cfg.n_samples:
                raise ValueError(f"x[{i}] must hold n_samples = {self.cfg.n_samples} values")
        arr = (c_void_p * self.Q)(*[_dptr(xi) for xi in xs])
        return arr, xs

    def _templates(self, templates):
        """(n_t, device templates [n_t, 5]): rows (a_p, T_asc, P, e, omega); [n_t, 3]
        circular rows are widened with e = omega = 0 (a device copy, ordered on the stream)."""
        import torch
        _check_tensor("templates", templates, torch.float64)
        if templates.dim() != 2 or templates.shape[1] not in (3, 5):
            raise ValueError("templates must be [n_t, 5] (a_p, T_asc, P, e, omega) or [n_t, 3] (circular)")
        return templates.shape[0], templates5(templates)

    # -- the C ABI calls -------------------------------------------------------
    def resample(self, x, templates, ab=None, norm=None, stream=None):
        """Stage 1: a_r, b_r series [n_t, Q, 2, N_tau] and segment norms [n_t, Q, M, 4]."""
        import torch
        n_t, templates = self._templates(templates)
        xp, _ = self._xptrs(x)
        dev = templates.device
        if ab is None:
            if self.store == STORE_BF16:
                ab = torch.empty((n_t, self.Q, 2, self.N_tau, 2), dtype=torch.bfloat16, device=dev)
            else:
                ab = torch.empty((n_t, self.Q, 2, self.N_tau), dtype=torch.complex64, device=dev)
        if norm is None:
            norm = torch.empty((n_t, self.Q, self.M, 4), dtype=torch.float32, device=dev)
        check("crosscorr_resample", self._lib.crosscorr_resample(
            self._h, xp, _dptr(templates), n_t, _dptr(ab), _dptr(norm), _stream_handle(stream)))
        return ab, norm

    def segment_fft(self, ab, n_t, F=None, stream=None):
        """Stage 2: spectra [n_t, Q, M, 2, N_f] complex64."""
        import torch
        if F is None:
            F = torch.empty((n_t, self.Q, self.M, 2, self.N_f), dtype=torch.complex64, device=ab.device)
        check("crosscorr_segment_fft", self._lib.crosscorr_segment_fft(
            self._h, _dptr(ab), n_t, _dptr(F), _stream_handle(stream)))
        return F

    def pair_accumulate(self, F, norm, n_t, rho=None, stream=None):
        """Stage 3: rho [n_t, N_f] float32."""
        import torch
        if rho is None:
            rho = torch.empty((n_t, self.N_f), dtype=torch.float32, device=F.device)
        check("crosscorr_pair_accumulate", self._lib.crosscorr_pair_accumulate(
            self._h, _dptr(F), _dptr(norm), n_t, _dptr(rho), _stream_handle(stream)))
        return rho

    def search(self, x, templates, rho=None, stream=None):
        """The whole path: rho [n_t, N_f] float32."""
        import torch
        n_t, templates = self._templates(templates)
        xp, _ = self._xptrs(x)
        if rho is None:
            rho = torch.empty((n_t, self.N_f), dtype=torch.float32, device=templates.device)
        else:
            _check_tensor("rho", rho, torch.float32)
        check("crosscorr_search", self._lib.crosscorr_search(
            self._h, xp, _dptr(templates), n_t, _dptr(rho), _stream_handle(stream)))
        return rho

    def set_path(self, path: int):
        """How search() computes rho: PATH_AUTO, PATH_FUSED, PATH_TWO_PASS or PATH_STAGED."""
        check("crosscorr_plan_set_path", self._lib.crosscorr_plan_set_path(self._h, int(path)))

    @property
    def search_path(self) -> int:
        """The path search() takes (PATH_FUSED, PATH_TWO_PASS or PATH_STAGED)."""
        v = ctypes.c_int()
        check("crosscorr_plan_search_path", self._lib.crosscorr_plan_search_path(self._h, byref(v)))
        return v.value

    def workspace_size(self, n_t: int) -> int:
        """Device bytes search() needs for n_t templates on its current path and tuning."""
        v = ctypes.c_size_t()
        check("crosscorr_plan_workspace_size", self._lib.crosscorr_plan_workspace_size(self._h, int(n_t), byref(v)))
        return v.value

    def set_workspace(self, ws=None):
        """Use a caller-owned device buffer (a CUDA uint8 tensor, kept alive here) as the
        search workspace; None returns to plan-owned memory."""
        import torch
        if ws is None:
            check("crosscorr_plan_set_workspace", self._lib.crosscorr_plan_set_workspace(self._h, None, 0))
            self._ws = None
            return
        _check_tensor("workspace", ws, torch.uint8)
        check("crosscorr_plan_set_workspace",
              self._lib.crosscorr_plan_set_workspace(self._h, c_void_p(_dptr(ws)), ws.numel()))
        self._ws = ws

    def set_tuning(self, batch_templates: int = 0, chunk_waves: int = 0, transform_len: int = 0):
        """Work split of search(): templates per two-pass batch, target CTA waves of the
        segment-chunk split, and the two-pass coset transform length (0: the plan's; 4096:
        the persistent kernel's, segments zero-padded) (0: defaults)."""
        t = CcTuning(int(batch_templates), int(chunk_waves), int(transform_len))
        check("crosscorr_plan_set_tuning", self._lib.crosscorr_plan_set_tuning(self._h, byref(t)))

    def demod_prepare(self, x, n_bin: int = 2, doppler_max: float = 0.0, stream=None):
        """Detector-frame (demodulation) search, step 1: SFTs of the locked T_sft blocks."""
        xp, self._demod_x = self._xptrs(x)
        check("crosscorr_demod_prepare", self._lib.crosscorr_demod_prepare(
            self._h, xp, int(n_bin), float(doppler_max), _stream_handle(stream)))

    def set_demod_form(self, separable: bool):
        """Pair sum of demod_search: the method's pair loop (default) or the separable
        window-sum form (the same rho up to FP32 rounding)."""
        check("crosscorr_plan_set_demod_form", self._lib.crosscorr_plan_set_demod_form(self._h, int(bool(separable))))

    def demod_search(self, templates, rho=None, stream=None):
        """Detector-frame (demodulation) rho [n_t, N_f] at the plan's output frequencies."""
        import torch
        n_t, templates = self._templates(templates)
        if rho is None:
            rho = torch.empty((n_t, self.N_f), dtype=torch.float32, device=templates.device)
        _check_tensor("rho", rho, torch.float32)
        check("crosscorr_demod_search", self._lib.crosscorr_demod_search(
            self._h, _dptr(templates), n_t, _dptr(rho), _stream_handle(stream)))
        return rho

    def set_kernel_timing(self, on: bool = True):
        """Diagnostic: bracket each launch of the search's dominant kernel (spectrum + pair
        sum on the two-pass path, the one-pass kernel on the fused path) with CUDA events."""
        check("crosscorr_plan_set_kernel_timing", self._lib.crosscorr_plan_set_kernel_timing(self._h, int(on)))

    def kernel_time(self):
        """(total ms, launches) of the dominant-kernel launches timed since the last call."""
        ms, n = c_double(), c_int64()
        check("crosscorr_plan_kernel_time", self._lib.crosscorr_plan_kernel_time(self._h, byref(ms), byref(n)))
        return ms.value, n.value

    def check(self, stream=None):
        """Synchronise the stream and raise if a kernel's bounded device wait ran out since
        the last check (the rho of those searches is then invalid)."""
        check("crosscorr_plan_check", self._lib.crosscorr_plan_check(self._h, _stream_handle(stream)))

    def set_wait_test(self, on: bool = True):
        """Diagnostic: make the persistent kernel's first bounded wait in every CTA run out
        (tests of the timeout path; the search's rho is then invalid)."""
        check("crosscorr_plan_set_wait_test", self._lib.crosscorr_plan_set_wait_test(self._h, int(on)))

    def topk(self, rho, k, stream=None):
        """k best (template, bin, freq, rho), descending, ties by (template, bin)."""
        import torch
        _check_tensor("rho", rho, torch.float32)
        n_t = rho.numel() // self.N_f
        n = min(k, n_t * self.N_f)
        hits = (CcHit * max(n, 1))()
        check("crosscorr_rho_topk", self._lib.crosscorr_rho_topk(
            self._h, _dptr(rho), n_t, k, hits, _stream_handle(stream)))
        out = np.zeros(n, dtype=[("tmpl", np.int64), ("bin", np.int32), ("freq", np.float64),
                                 ("rho", np.float32)])
        for i in range(n):
            out[i] = (hits[i].tmpl, hits[i].bin, hits[i].freq, hits[i].rho)
        return out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.crosscorr_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
