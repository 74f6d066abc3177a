"""Seeded synthetic inputs for the time-domain Lienard-Wiechert path.

This package generates electron trajectories (t, r, beta, beta_dot), detector
directions and named workload configurations.  It contains none of the
radiation method's arithmetic (no advanced times, fields, deposits or
transforms), so both the CPU oracle and the CUDA library can consume its
output without sharing code.  All randomness comes from
``numpy.random.Generator(PCG64(seed))``.
"""
from .physics import C0, Q_E, M_E, EPS0  # noqa: F401
from .detector import detector_grid, detector_ring  # noqa: F401
from .planewave import plane_wave_trajectories  # noqa: F401
from .boris import GaussianLaser, boris_trajectories, gaussian_bunch  # noqa: F401
from .simple import (  # noqa: F401
    Trajectories,
    stationary_constant_acceleration,
    linear_ramp_acceleration,
    uniform_motion,
    circular_motion,
    random_smooth,
)
from . import configs  # noqa: F401
