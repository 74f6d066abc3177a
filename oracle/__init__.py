"""FP64 CPU oracle for the time-domain Lienard-Wiechert path (arXiv 2206.03015).

TEST INFRASTRUCTURE ONLY: this package is the slow, obviously-correct
reference that the CUDA library is checked against.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with ``paper_2206_03015_gb300`` and never imports it.
"""
from .oracle import (  # noqa: F401
    build,
    load,
    grid_bounds,
    advanced_times,
    fields,
    tdm_deposit,
    fft,
    dft,
    spectrum,
    fdm,
    tdm_grad,
    num_threads,
    FLAG_ACCEL,
    FLAG_VELOCITY,
    FLAG_EXACT,
    ST_BETA,
    ST_NONFINITE,
    ST_TIME,
    ST_CLIP,
    ST_TA_ORDER,
)
from . import estimates  # noqa: F401
