"""GPU frequency-domain method (Eq. inty_dft) against the CPU oracle's FDM, and
the time-domain path against the GPU FDM on a Nyquist-resolved beam (the
paper's TDM/FDM comparison, normalised error of Eq. spectra_error)."""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_cases import rel_l2
from paper_2206_03015_gb300 import lw
from workloads import configs
from workloads.planewave import doppler_fundamental, plane_wave_trajectories

pytestmark = pytest.mark.gpu


def _dirs(n, seed, max_angle):
    rng = np.random.Generator(np.random.PCG64(seed))
    tx = rng.uniform(-max_angle, max_angle, n)
    ty = rng.uniform(-max_angle, max_angle, n)
    return np.stack([np.sin(tx), np.cos(tx) * np.sin(ty), np.cos(tx) * np.cos(ty)], -1)


@pytest.mark.parametrize("n_omega", [1, 1000, 2500])
def test_fdm_matches_oracle(n_omega):
    g = 5.0
    tr = plane_wave_trajectories(g, 1e-6, 0.3, 20e-15, -50e-15, 50e-15, 700, n_e=2,
                                 z_offsets=[0.0, 3e-7])
    n_hat = _dirs(3, 4, 0.5 / g)
    w1 = doppler_fundamental(g, 1e-6, 0.3)
    # one frequency: the fundamental.  A lone point far below it (0.2 w1) lies where
    # the sum cancels almost completely, so its relative error measures the
    # cancellation, not the kernel: FP32 twiddles leave ~1e-7 of the summed terms.
    omega0, d_omega = (w1, 0.0) if n_omega == 1 else (0.2 * w1, 2.5 * w1 / n_omega)
    dt = float(tr.t[1] - tr.t[0])
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot, sections=lw.LW_SECTION_FP64)
    S = lw.lw_spectrum_fdm(traj, lw.Detector(n_hat), omega0, d_omega, n_omega, dt).cpu().numpy()
    om = omega0 + d_omega * np.arange(n_omega)
    S_o, _ = oracle.fdm(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, om, dt)
    assert rel_l2(S, S_o) <= 1e-5


def test_tdm_and_fdm_agree_on_resolved_beam():
    # 2^16 bins: Nyquist above the second harmonic, so no harmonic aliases into the band
    w = configs.c2x(n_e=32, n_s=3000, nx=4, n_bins=1 << 16)
    tr = w.traj
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot)
    det = lw.Detector(w.n_hat)
    b = lw.lw_grid_bounds(traj, det).cpu().numpy()
    grid = lw.grid_from_bounds(b[0], b[1], w.n_bins)
    rec = lw.lw_deposit_time_domain(traj, det, grid, lw.LW_FP64)
    S_t = lw.lw_spectrum(rec, lw.LW_FP64, det.n_pix, grid).cpu().numpy()
    d_omega = 2 * math.pi / (grid.n_bins * grid.dt_u)
    w1 = doppler_fundamental(w.gamma, w.lam, w.a0)
    l0 = int(0.6 * w1 / d_omega)
    n_om = int(0.8 * w1 / d_omega)
    S_f = lw.lw_spectrum_fdm(traj, det, l0 * d_omega, d_omega, n_om,
                             float(tr.t[1] - tr.t[0])).cpu().numpy()
    err = np.abs(S_t[:, l0:l0 + n_om] - S_f) / S_f.max()
    assert err.mean() < 1e-2 and err.max() < 0.13, (err.mean(), err.max())
