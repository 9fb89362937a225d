"""FP64 CPU oracle of the resampled CrossCorr statistic (TEST INFRASTRUCTURE).

This package is the independent reference that the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it; the product path never
does, and it shares no code with the CUDA library (only the seeded input
generator in ``synth`` serves both sides).

Every function cites the passage of the paper it follows.  Parity status:
all functions are pinned by ``tests/test_oracle_pins.py``.  The learned
interpolator (``oracle.learned``) is PARITY UNPINNED against the paper, which has no
such component; it is pinned by tone reproduction and judged against the exact
stencil.
"""
from . import learned  # noqa: F401
from .crosscorr import (  # noqa: F401
    PAIR_UNORDERED, PAIR_CROSS_ONLY, PAIR_ALL_ORDERED,
    Plan, make_plan, ssb_delay, delay, stencil_position, interpolate, hamming, timing,
    periapsis_time, kepler_E, binary_delay, orbit,
    resample, noise_block,
    weights, spectra_direct, spectra_fft, segment_norms, pair_list,
    normalization, pair_sum, rho_template, rho, topk, detector_frame_rho,
)
