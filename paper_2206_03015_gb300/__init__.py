"""GB300-native time-domain Lienard-Wiechert radiation spectra (arXiv 2206.03015).

The compute path is liblw.so (hand-written CUDA for sm_103a, C ABI in
include/lw.h); ``lw`` is its thin Python binding.
"""
from . import lw  # noqa: F401
from .lw import (  # noqa: F401
    Detector,
    Grid,
    LW_FIELD_ACCEL,
    LW_FIELD_VELOCITY,
    LW_FP64,
    LW_MIXED,
    LW_MIXED_KAHAN,
    LW_MIXED_F32,
    LW_MIXED_F32X4,
    LW_SECTION_FP64,
    LW_SECTION_MIXED,
    grid_from_bounds,
    lw_deposit_time_domain,
    lw_grid_bounds,
    lw_spectrum,
    lw_trajectories_upload,
)
