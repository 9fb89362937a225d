"""The C ABI library builds, loads and exports every symbol the header declares;
host-side argument validation rejects bad input before any CUDA call.  No
compute calls: these run without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from paper_1712_06515_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "crosscorr.h")

CC_OK, CC_ERR_INVALID, CC_ERR_UNSUPPORTED = 0, 1, 5


@pytest.fixture(scope="module")
def lib():
    _lib.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(crosscorr_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("crosscorr_plan", "crosscorr_plan_info", "crosscorr_resample",
                     "crosscorr_segment_fft", "crosscorr_pair_accumulate", "crosscorr_search",
                     "crosscorr_rho_topk", "crosscorr_plan_destroy", "crosscorr_status_string",
                     "crosscorr_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, name


def test_struct_layouts_match_header():
    # sizes of the ABI structs as laid out by a C compiler for this header
    assert ctypes.sizeof(_lib.CcConfig) == 8 * 8 + 6 * 4 + 8
    assert ctypes.sizeof(_lib.CcDetector) == 11 * 8
    assert ctypes.sizeof(_lib.CcHit) == 32
    assert ctypes.sizeof(_lib.CcPlanInfo) == 9 * 8 + 7 * 8 + 8
    assert ctypes.sizeof(_lib.CcTuning) == 16
    assert ctypes.sizeof(_lib.CcLearnedInterp) == 40


def _cfg(**kw):
    ds = synth.tiny()
    c = _lib.CcConfig()
    for f in ("t0", "dt", "f_h", "f_band", "T_sft", "T_short", "T_max", "mu_f", "D", "pair_mode"):
        setattr(c, f, getattr(ds.cfg, f))
    c.n_det, c.interp, c.store, c.n_samples = 2, 0, 0, ds.cfg.n_samples
    for k, v in kw.items():
        setattr(c, k, v)
    return c, ds


def _dets(ds, mutate=None):
    keep, arr = [], (_lib.CcDetector * 2)()
    for i, d in enumerate(ds.dets):
        tabs = [np.ascontiguousarray(v, np.float64) for v in (d.ssb_delay, d.a_tab, d.b_tab, d.sigma)]
        if mutate:
            mutate(i, tabs)
        keep += tabs
        P = ctypes.POINTER(ctypes.c_double)
        arr[i].ssb_delay, arr[i].eph_t0, arr[i].eph_dt, arr[i].n_eph = (
            tabs[0].ctypes.data_as(P), d.eph_t0, d.eph_dt, tabs[0].size)
        arr[i].a_tab, arr[i].b_tab = tabs[1].ctypes.data_as(P), tabs[2].ctypes.data_as(P)
        arr[i].ab_t0, arr[i].ab_dt, arr[i].n_ab = d.ab_t0, d.ab_dt, tabs[1].size
        arr[i].sigma, arr[i].n_sigma = tabs[3].ctypes.data_as(P), tabs[3].size
    return arr, keep


BAD_CONFIGS = [
    dict(n_det=0), dict(n_det=5), dict(D=0), dict(D=33), dict(dt=0.0), dict(n_samples=0),
    dict(f_band=0.0), dict(f_band=1.5), dict(mu_f=0.0), dict(T_max=-1.0), dict(pair_mode=3),
    dict(store=2), dict(interp=7), dict(T_sft=0.5), dict(T_short=127.5), dict(n_samples=100),
]


@pytest.mark.parametrize("kw", BAD_CONFIGS)
def test_plan_rejects_bad_config(lib, kw):
    c, ds = _cfg(**kw)
    arr, keep = _dets(ds)
    h = ctypes.c_void_p()
    st = lib.crosscorr_plan(ctypes.byref(c), arr, ctypes.byref(h))
    assert st == CC_ERR_INVALID, (kw, st, lib.crosscorr_last_error())
    assert lib.crosscorr_last_error()
    assert not h.value


def test_plan_accepts_learned_interp(lib):
    # interp = LEARNED passes validation; without a GPU the plan then stops at its
    # first device upload (CC_ERR_CUDA), with a GPU it is built
    c, ds = _cfg(interp=1)
    arr, keep = _dets(ds)
    h = ctypes.c_void_p()
    st = lib.crosscorr_plan(ctypes.byref(c), arr, ctypes.byref(h))
    assert st in (CC_OK, 3), (st, lib.crosscorr_last_error())
    lib.crosscorr_plan_destroy(h)


def test_set_learned_interp_rejects_null(lib):
    li = _lib.CcLearnedInterp()
    assert lib.crosscorr_plan_set_learned_interp(None, ctypes.byref(li)) == CC_ERR_INVALID
    assert lib.crosscorr_plan_set_learned_interp(None, None) == CC_ERR_INVALID
    assert ctypes.sizeof(_lib.CcLearnedInterp) == 5 * 8


@pytest.mark.parametrize("which", ["neg_sigma", "nan_ssb", "nan_a"])
def test_plan_rejects_bad_tables(lib, which):
    def mutate(i, tabs):
        if i == 1:
            if which == "neg_sigma":
                tabs[3][5] = -1.0
            elif which == "nan_ssb":
                tabs[0][3] = np.nan
            else:
                tabs[1][2] = np.inf
    c, ds = _cfg()
    arr, keep = _dets(ds, mutate)
    h = ctypes.c_void_p()
    assert lib.crosscorr_plan(ctypes.byref(c), arr, ctypes.byref(h)) == CC_ERR_INVALID


def test_entry_points_reject_null_plan(lib):
    assert lib.crosscorr_resample(None, None, None, 1, None, None, None) == CC_ERR_INVALID
    assert lib.crosscorr_segment_fft(None, None, 1, None, None) == CC_ERR_INVALID
    assert lib.crosscorr_pair_accumulate(None, None, None, 1, None, None) == CC_ERR_INVALID
    assert lib.crosscorr_search(None, None, None, 1, None, None) == CC_ERR_INVALID
    hits = (_lib.CcHit * 1)()
    assert lib.crosscorr_rho_topk(None, None, 1, 1, hits, None) == CC_ERR_INVALID
    assert lib.crosscorr_plan_set_kernel_timing(None, 1) == CC_ERR_INVALID
    assert lib.crosscorr_plan_set_path(None, 0) == CC_ERR_INVALID
    assert lib.crosscorr_plan_set_workspace(None, None, 0) == CC_ERR_INVALID
    t = _lib.CcTuning(0, 0, 0)
    assert lib.crosscorr_plan_set_tuning(None, ctypes.byref(t)) == CC_ERR_INVALID
    nb = ctypes.c_size_t()
    assert lib.crosscorr_plan_workspace_size(None, 1, ctypes.byref(nb)) == CC_ERR_INVALID
    pth = ctypes.c_int()
    assert lib.crosscorr_plan_search_path(None, ctypes.byref(pth)) == CC_ERR_INVALID
    ms, n = ctypes.c_double(), ctypes.c_int64()
    assert lib.crosscorr_plan_kernel_time(None, ctypes.byref(ms), ctypes.byref(n)) == CC_ERR_INVALID
    lib.crosscorr_plan_destroy(None)
    assert lib.crosscorr_status_string(3) == b"CUDA error"
