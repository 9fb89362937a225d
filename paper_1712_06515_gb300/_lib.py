"""Build and load the crosscorr CUDA library (libcrosscorr.so) and declare its C ABI.

The library is compiled in-tree for sm_103a with nvcc; nothing here computes any
part of the statistic.  Loading fails loudly when the library is missing or
stale, so no caller can silently run without the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from ctypes import POINTER, c_double, c_float, c_int, c_int32, c_int64, c_size_t, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIBPATH = os.path.join(LIBDIR, "libcrosscorr.so")

SOURCES = ["plan.cu", "stages.cu", "search.cu", "topk.cu", "fused.cu", "fused_l64_256.cu", "fused_l512_1024.cu",
           "fused_l2048.cu", "fused_l4096.cu", "noalloc.cu", "learned.cu", "segpair.cu", "segpair_tma.cu", "peak.cu", "demod.cu", "sftseries.cu", "lattice.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "crosscorr.h"))
    return files


def is_stale() -> bool:
    if not os.path.exists(LIBPATH):
        return True
    t = os.path.getmtime(LIBPATH)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libcrosscorr.so."""
    if not force and not is_stale():
        return LIBPATH
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIBPATH + ".tmp"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp,
                        *objs, "-ldl"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIBPATH)
    return LIBPATH


# ---------------------------------------------------------------------------
# ABI structures (mirror include/crosscorr.h)
# ---------------------------------------------------------------------------
class CcConfig(ctypes.Structure):
    _fields_ = [("t0", c_double), ("dt", c_double), ("f_h", c_double), ("f_band", c_double),
                ("T_sft", c_double), ("T_short", c_double), ("T_max", c_double), ("mu_f", c_double),
                ("n_det", c_int32), ("D", c_int32), ("interp", c_int32), ("store", c_int32),
                ("pair_mode", c_int32), ("reserved", c_int32), ("n_samples", c_int64)]


class CcDetector(ctypes.Structure):
    _fields_ = [("ssb_delay", POINTER(c_double)), ("eph_t0", c_double), ("eph_dt", c_double),
                ("n_eph", c_int64), ("a_tab", POINTER(c_double)), ("b_tab", POINTER(c_double)),
                ("ab_t0", c_double), ("ab_dt", c_double), ("n_ab", c_int64),
                ("sigma", POINTER(c_double)), ("n_sigma", c_int64)]


class CcHit(ctypes.Structure):
    _fields_ = [("tmpl", c_int64), ("bin", c_int32), ("pad", c_int32), ("freq", c_double),
                ("rho", c_float), ("pad2", c_float)]


class CcPlanInfo(ctypes.Structure):
    _fields_ = [("N_s", c_int64), ("M", c_int64), ("R", c_int64), ("N_tau", c_int64),
                ("N_FFT", c_int64), ("N_f", c_int64), ("k0", c_int64), ("L", c_int64), ("C", c_int64),
                ("T_coh", c_double), ("dlf", c_double), ("N_FFT0", c_double), ("T_FFT", c_double),
                ("nu_R", c_double), ("f_r", c_double), ("f_FFT", c_double), ("ws_bytes", c_size_t)]


class CcLearnedInterp(ctypes.Structure):
    _fields_ = [("weights_bf16", POINTER(ctypes.c_uint16)), ("n_weights", c_int64),
                ("nu_lo", c_double), ("nu_hi", c_double), ("nu_c", c_double)]


class CcTuning(ctypes.Structure):
    _fields_ = [("batch_templates", c_int64), ("chunk_waves", c_int32), ("transform_len", c_int32)]


# every symbol the header declares, with its signature
SIGNATURES = {
    "crosscorr_plan": (c_int, [POINTER(CcConfig), POINTER(CcDetector), POINTER(c_void_p)]),
    "crosscorr_plan_info": (c_int, [c_void_p, POINTER(CcPlanInfo), POINTER(c_double), POINTER(c_int64)]),
    "crosscorr_plan_set_learned_interp": (c_int, [c_void_p, POINTER(CcLearnedInterp)]),
    "crosscorr_resample": (c_int, [c_void_p, POINTER(c_void_p), c_void_p, c_int64, c_void_p, c_void_p,
                                   c_void_p]),
    "crosscorr_segment_fft": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "crosscorr_pair_accumulate": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "crosscorr_search": (c_int, [c_void_p, POINTER(c_void_p), c_void_p, c_int64, c_void_p, c_void_p]),
    "crosscorr_search_noalloc": (c_int, [c_void_p, POINTER(c_void_p), c_void_p, c_int64, c_void_p,
                                         c_void_p]),
    "crosscorr_rho_topk": (c_int, [c_void_p, c_void_p, c_int64, c_int, POINTER(CcHit), c_void_p]),
    "crosscorr_plan_destroy": (None, [c_void_p]),
    "crosscorr_status_string": (ctypes.c_char_p, [c_int]),
    "crosscorr_last_error": (ctypes.c_char_p, []),
    "crosscorr_kernel_launches": (ctypes.c_uint64, []),
    "crosscorr_plan_set_kernel_timing": (c_int, [c_void_p, c_int]),
    "crosscorr_plan_set_path": (c_int, [c_void_p, c_int]),
    "crosscorr_demod_prepare": (c_int, [c_void_p, POINTER(c_void_p), c_int32, c_double, c_void_p]),
    "crosscorr_metric": (c_int, [c_double, c_double, c_double, c_int32, c_double, c_void_p, c_double,
                                 POINTER(c_double)]),
    "crosscorr_lattice": (c_int, [POINTER(c_double), c_double, POINTER(c_double), POINTER(c_double), c_void_p,
                                  c_int64, POINTER(c_int64)]),
    "crosscorr_sfts_to_series": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_double, c_double, c_void_p,
                                         c_void_p]),
    "crosscorr_demod_search": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "crosscorr_plan_set_demod_form": (c_int, [c_void_p, c_int]),
    "crosscorr_plan_set_workspace": (c_int, [c_void_p, c_void_p, c_size_t]),
    "crosscorr_plan_workspace_size": (c_int, [c_void_p, c_int64, POINTER(c_size_t)]),
    "crosscorr_plan_set_tuning": (c_int, [c_void_p, POINTER(CcTuning)]),
    "crosscorr_plan_search_path": (c_int, [c_void_p, POINTER(c_int)]),
    "crosscorr_plan_kernel_time": (c_int, [c_void_p, POINTER(c_double), POINTER(c_int64)]),
    "crosscorr_plan_check": (c_int, [c_void_p, c_void_p]),
    "crosscorr_plan_set_wait_test": (c_int, [c_void_p, c_int]),
    "crosscorr_measure_fp32_peak": (c_int, [POINTER(c_double), c_void_p]),
}

_LIB = None


def load(path: str = LIBPATH) -> ctypes.CDLL:
    """Load the compiled library; raises if it is missing or older than its sources."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"crosscorr CUDA library not built ({path}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    if path == LIBPATH and is_stale():
        raise ImportError("crosscorr CUDA library is older than its sources; rebuild it")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class CrossCorrError(RuntimeError):
    def __init__(self, call: str, status: int):
        lib = load()
        msg = lib.crosscorr_status_string(status).decode()
        detail = lib.crosscorr_last_error().decode()
        super().__init__(f"{call}: {msg} ({status}): {detail}")
        self.status = status


def check(call: str, status: int) -> None:
    if status != 0:
        raise CrossCorrError(call, status)
