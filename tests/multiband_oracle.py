"""Oracle rho of the multi-band workload, band by band in a spawned process pool (the
GPU tests call this after CUDA is initialised, so workers must not be forked)."""
import dataclasses
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import oracle
import synth


def oracle_band(args):
    b, per_band, D = args
    ds = synth.multiband_band(b, max_templates=per_band)
    if D is not None:
        ds = dataclasses.replace(ds, cfg=dataclasses.replace(ds.cfg, D=D))
    return oracle.rho(ds)


def oracle_all(n_bands, per_band, D=None):
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=ctx) as ex:
        return list(ex.map(oracle_band, [(b, per_band, D) for b in range(n_bands)]))
