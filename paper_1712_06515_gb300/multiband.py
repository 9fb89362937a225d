"""Batched multi-band search: many bands (each its own plan, series and template grid)
run back to back from one CUDA graph launch.

Every band's `crosscorr_search` is recorded once into a CUDA graph; replaying the graph
launches all bands' kernels with one host call.  The plans share one caller-owned
workspace (their searches run in order on one stream), sized for the largest band, so
nothing is allocated while the graph is captured or replayed.  Before capture an
autotuner picks, per band, the search path and the segment-chunk split with the best
measured time on a sample of that band's templates.

Argument marshalling and scheduling only: all arithmetic runs in the CUDA library.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from . import (INTERP_EXACT, PATH_FUSED, PATH_TWO_PASS, STORE_FP32, CrossCorrError, CrossCorrPlan, templates5)

CHUNK_WAVES = (5, 10, 20, 40, 80)


def autotune(plan: CrossCorrPlan, x, templates, reps: int = 2, chunk_waves: Sequence[int] = CHUNK_WAVES,
             stream=None) -> dict:
    """Time every (path, transform length, chunk split) the plan supports on `templates`
    and keep the fastest.  The transform length is the tile shape of the two-pass
    spectrum kernel: the plan's own coset length, or 4096-point cosets (the persistent
    kernel) with the segments zero-padded when the plan's cosets are shorter.

    Returns {"path", "transform_len", "chunk_waves", "ms"} of the choice and leaves the
    plan set to it."""
    import torch
    stream = stream or torch.cuda.current_stream()
    rho = torch.empty((templates.shape[0], plan.N_f), dtype=torch.float32, device=templates.device)
    best = None
    lens = (0, 4096) if plan.info["L"] < 4096 <= plan.info["N_FFT"] else (0,)
    for path in (PATH_TWO_PASS, PATH_FUSED):
        try:
            plan.set_path(path)
        except CrossCorrError:
            continue
        for tl in (lens if path == PATH_TWO_PASS else (0,)):
            for w in chunk_waves:
                plan.set_tuning(chunk_waves=w, transform_len=tl)
                plan.search(x, templates, rho, stream=stream)        # warm-up (workspace, caches)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    plan.search(x, templates, rho, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1) / reps
                if best is None or ms < best["ms"]:
                    best = {"path": path, "transform_len": tl, "chunk_waves": w, "ms": ms}
    if best is None:
        raise CrossCorrError("crosscorr_plan_set_path", 5)
    plan.set_path(best["path"])
    plan.set_tuning(chunk_waves=best["chunk_waves"], transform_len=best["transform_len"])
    return best


class MultiBandSearch:
    """rho of every band's templates, from one CUDA graph launch per run().

    bands: sequence of (cfg, dets, x, templates) with x a CUDA complex64 tensor
    [Q, N_t] and templates a CUDA float64 tensor [n_t, 3] (both kept resident)."""

    def __init__(self, bands: Sequence, store: int = STORE_FP32, interp: int = INTERP_EXACT,
                 tune: bool = True, tune_templates: int = 64, learned_weights: Optional[str] = None):
        import torch
        self.x = [b[2] for b in bands]
        self.templates = [templates5(b[3]) for b in bands]
        self.plans: List[CrossCorrPlan] = [
            CrossCorrPlan(cfg, dets, store=store, interp=interp, learned_weights=learned_weights)
            for cfg, dets, _, _ in bands]
        dev = self.templates[0].device
        self.rho = [torch.empty((t.shape[0], p.N_f), dtype=torch.float32, device=dev)
                    for p, t in zip(self.plans, self.templates)]
        self.tuning = []
        for p, x, t in zip(self.plans, self.x, self.templates):
            if tune:
                self.tuning.append(autotune(p, x, t[:tune_templates]))
            else:
                self.tuning.append({"path": p.search_path, "transform_len": 0, "chunk_waves": 0, "ms": None})
        # one shared workspace for the whole batch of bands
        need = max(p.workspace_size(t.shape[0]) for p, t in zip(self.plans, self.templates))
        self.workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
        for p in self.plans:
            p.set_workspace(self.workspace)
        self.graph = None
        self.kernels_per_run = 0

    @property
    def units(self) -> int:
        """template x bin values produced per run()."""
        return int(sum(r.numel() for r in self.rho))

    def _launch_all(self, stream=None):
        for p, x, t, r in zip(self.plans, self.x, self.templates, self.rho):
            p.search(x, t, r, stream=stream)

    def capture(self):
        """Run once (warm-up) and record every band's search into one CUDA graph."""
        import torch
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._launch_all(side)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        from . import _lib
        lib = _lib.load()
        g = torch.cuda.CUDAGraph()
        n0 = lib.crosscorr_kernel_launches()
        with torch.cuda.graph(g):
            self._launch_all()
        self.kernels_per_run = int(lib.crosscorr_kernel_launches() - n0)   # kernel nodes in the graph
        self.graph = g
        return self

    def run(self):
        """All bands' rho (in self.rho): one graph launch, or eager launches before capture()."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._launch_all()
        return self.rho

    def topk(self, k: int) -> List[np.ndarray]:
        """Per band, the k best (template, bin, freq, rho) records."""
        return [p.topk(r, k) for p, r in zip(self.plans, self.rho)]

    def close(self):
        for p in self.plans:
            p.close()
        self.plans = []
