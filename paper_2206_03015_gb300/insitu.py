"""In-situ time-domain spectra (Algorithm 2 as written: the trajectory update
sits inside the step loop).  The GPU Boris pusher produces the trajectories
one block of ``block_steps`` steps at a time; each block (with the last
sample of the previous block as its first sample) is deposited at once and
then overwritten, so memory holds one block instead of whole trajectories.
Block boundaries reuse the exact FP64 end-sample bins of the deposit, so
consecutive blocks neither drop nor double a grid point; in FP64 the result
equals the deposit of the stored trajectories up to summation order.
"""
from __future__ import annotations

import math

import torch

from . import lw


def grid_bounds_from_ends(t0, t1, r0, r1, det: "lw.Detector"):
    """Eqs. (tu_min), (tu_max) from the first and last positions only."""
    dev = r0.device
    n_e = r0.shape[0]
    t = torch.tensor([t0, t1], dtype=torch.float64, device=dev)
    r = torch.stack([r0, r1], 1).contiguous()
    zeros = torch.zeros_like(r)
    traj = lw.lw_trajectories_upload(t, r, zeros, zeros, sections=lw.LW_SECTION_FP64,
                                     device=dev)
    b = lw.lw_grid_bounds(traj, det).cpu().tolist()
    del n_e
    return b[0], b[1]


def in_situ_spectrum(r0, u0, laser, t_start: float, t_end: float, n_steps: int,
                     det: "lw.Detector", n_bins: int, precision: int = lw.LW_MIXED,
                     block_steps: int = 1024, grid: "lw.Grid | None" = None,
                     q: float = lw.Q_E, anchor_block: int = 512):
    """Spectra S [n_pix][n_bins/2+1] of electrons starting at (r0, u0) ([n_e, 3] float64 CUDA
    tensors; u = gamma beta) in the Gaussian laser (lam, a0, w0, fwhm).  Without ``grid`` the
    observer grid comes from a trial push (Eqs. tu_min / tu_max of the first and last
    positions).  Returns (S, grid, record)."""
    dev = r0.device
    n_e = r0.shape[0]
    dt = (t_end - t_start) / n_steps
    B = int(min(block_steps, n_steps))
    t_b = torch.empty(B + 1, dtype=torch.float64, device=dev)
    bufs = [torch.empty(n_e * (B + 1) * 3, dtype=torch.float64, device=dev) for _ in range(3)]
    if grid is None:                  # trial push: final positions only
        r, u = r0.clone(), u0.clone()
        for s0 in range(0, n_steps, B):
            nb = min(B, n_steps - s0)
            lw.lw_boris_push(r, u, t_start, dt, nb, laser, t_b, *bufs, step0=s0)
        lo, hi = grid_bounds_from_ends(t_start, t_start + n_steps * dt, r0, r, det)
        grid = lw.grid_from_bounds(lo, hi, n_bins)
    shp, dtype = lw.record_shape(det, grid, precision)
    record = torch.zeros(shp, dtype=dtype, device=dev)
    r, u = r0.clone(), u0.clone()
    sections = lw.LW_SECTION_FP64 if precision == lw.LW_FP64 else lw.LW_SECTION_MIXED
    ws = None
    for s0 in range(0, n_steps, B):
        nb = min(B, n_steps - s0)
        lw.lw_boris_push(r, u, t_start, dt, nb, laser, t_b, *bufs, step0=s0)
        views = [x[: n_e * (nb + 1) * 3].view(n_e, nb + 1, 3) for x in bufs]
        traj = lw.lw_trajectories_upload(t_b[: nb + 1], *views, sections=sections,
                                         block=anchor_block, device=dev, ws=ws)
        ws = traj.ws
        lw.lw_deposit_time_domain(traj, det, grid, precision, record=record, accumulate=True)
    S = lw.lw_spectrum(record, precision, det.n_pix, grid, q=q)
    return S, grid, record


def t_u_estimate(l_x: float, l_y: float, l_z: float, T_laser: float, gamma: float,
                 c0: float = 299792458.0) -> float:
    """Eq. (Tu_estimation): T_u ~ l_x/(gamma c0) + l_y/(gamma c0) + l_z/c0 + T_laser/(2 gamma^2),
    the grid length the paper uses when no trial push is made."""
    return (l_x / (gamma * c0) + l_y / (gamma * c0) + l_z / c0
            + T_laser / (2.0 * gamma * gamma))


def n_tu_estimate(t_u: float, gamma: float, lam0: float, c0: float = 299792458.0) -> int:
    """Eqs. (NTu_estimation_1..3): N_Tu = 2 omega_max / d_omega with omega_max = 4 gamma^2
    omega_0 and d_omega = 2 pi / T_u, rounded up to a power of two for the FFT."""
    omega0 = 2.0 * math.pi * c0 / lam0
    n = 2.0 * 4.0 * gamma * gamma * omega0 / (2.0 * math.pi / t_u)
    return 1 << max(1, math.ceil(math.log2(n)))
