"""In-situ path (GPU Boris pusher + block-wise deposit): the pusher matches the
workload generator's pusher, block-wise deposition equals deposition of the
stored trajectories (FP64: up to summation order; mixed: to 1e-4), and the
in-situ spectra match the oracle's deposit + spectrum of the same motion."""
import numpy as np
import pytest
import torch

import oracle
from gpu_cases import rel_l2
from paper_2206_03015_gb300 import lw
from paper_2206_03015_gb300.insitu import in_situ_spectrum
from workloads.boris import GaussianLaser, boris_trajectories, gaussian_bunch

pytestmark = pytest.mark.gpu


def _beam(n_e=24, n_s=1500):
    laser = GaussianLaser(lam=0.8e-6, a0=0.5, w0=20e-6, fwhm=30e-15)
    t_half = 60e-15
    r0, u0 = gaussian_bunch(n_e, 77, 0.5e-6, 0.5e-6, 0.1e-6, 60.0, 1e-3, 0.5e-6, -t_half)
    return laser, r0, u0, -t_half, t_half, n_s


def test_gpu_pusher_matches_generator():
    laser, r0, u0, t0, t1, n_s = _beam(n_s=800)
    ref = boris_trajectories(r0, u0, laser, t0, t1, n_s)
    r = torch.from_numpy(r0).cuda()
    u = torch.from_numpy(u0).cuda()
    n_e = r0.shape[0]
    t = torch.empty(n_s + 1, dtype=torch.float64, device="cuda")
    out = [torch.empty((n_e, n_s + 1, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    lw.lw_boris_push(r, u, t0, (t1 - t0) / n_s, n_s, (laser.lam, laser.a0, laser.w0, laser.fwhm),
                     t, *out)
    torch.cuda.synchronize()
    assert np.max(np.abs(t.cpu().numpy() - ref.t)) <= 1e-27
    assert np.max(np.abs(out[0].cpu().numpy() - ref.r)) <= 1e-10 * np.abs(ref.r).max()
    assert np.max(np.abs(out[1].cpu().numpy() - ref.beta)) <= 1e-10
    assert np.max(np.abs(out[2].cpu().numpy() - ref.beta_dot)) <= 1e-8 * np.abs(ref.beta_dot).max()


@pytest.mark.parametrize("precision,tol", [(lw.LW_FP64, 1e-12), (lw.LW_MIXED, 1e-4)])
def test_block_wise_deposit_equals_stored_trajectories(precision, tol):
    laser, r0, u0, t0, t1, n_s = _beam()
    L = (laser.lam, laser.a0, laser.w0, laser.fwhm)
    rng = np.random.Generator(np.random.PCG64(5))
    tx, ty = rng.uniform(-0.02, 0.02, 9), rng.uniform(-0.02, 0.02, 9)
    det = lw.Detector(np.stack([np.sin(tx), np.cos(tx) * np.sin(ty), np.cos(tx) * np.cos(ty)], -1))
    r = torch.from_numpy(r0).cuda()
    u = torch.from_numpy(u0).cuda()
    S_blk, grid, _ = in_situ_spectrum(r, u, L, t0, t1, n_s, det, 1 << 14, precision=precision,
                                      block_steps=256)
    # stored: the whole trajectory from one push
    n_e = r0.shape[0]
    t = torch.empty(n_s + 1, dtype=torch.float64, device="cuda")
    out = [torch.empty((n_e, n_s + 1, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    lw.lw_boris_push(r.clone(), u.clone(), t0, (t1 - t0) / n_s, n_s, L, t, *out)
    traj = lw.lw_trajectories_upload(t, *out)
    rec = lw.lw_deposit_time_domain(traj, det, grid, precision)
    S = lw.lw_spectrum(rec, precision, det.n_pix, grid)
    torch.cuda.synchronize()
    assert rel_l2(S_blk.double().cpu().numpy(), S.double().cpu().numpy()) <= tol


def _oracle_spectrum(t, r, beta, bdot, n_hat, grid):
    rec, st = oracle.tdm_deposit(t, r, beta, bdot, n_hat, grid.t_min, grid.dt_u, grid.n_bins)
    return oracle.spectrum(rec, grid.dt_u), st


@pytest.mark.parametrize("precision", [lw.LW_FP64, lw.LW_MIXED, lw.LW_MIXED_F32])
def test_in_situ_matches_oracle(precision):
    """Algorithm 2 as written (trajectory update inside the step loop), checked against
    the definition: the in-situ spectrum of one initial state against the oracle's
    deposit + spectrum of (a) the samples the GPU pusher produced, read back to the host
    (same inputs: FP64 1e-9, mixed 1e-4), and (b) the trajectories of the workload's own
    numpy Boris pusher from the same initial state (independent of every GPU kernel: the
    two pushers differ by rounding, <= 1e-8 relative in beta_dot, so FP64 within 1e-6)."""
    laser, r0, u0, t0, t1, n_s = _beam(n_e=12, n_s=1200)
    L = (laser.lam, laser.a0, laser.w0, laser.fwhm)
    rng = np.random.Generator(np.random.PCG64(11))
    tx, ty = rng.uniform(-0.02, 0.02, 7), rng.uniform(-0.02, 0.02, 7)
    n_hat = np.stack([np.sin(tx), np.cos(tx) * np.sin(ty), np.cos(tx) * np.cos(ty)], -1)
    det = lw.Detector(n_hat)
    r = torch.from_numpy(r0).cuda()
    u = torch.from_numpy(u0).cuda()
    S_gpu, grid, _ = in_situ_spectrum(r, u, L, t0, t1, n_s, det, 1 << 13, precision=precision,
                                      block_steps=200)
    S_gpu = S_gpu.double().cpu().numpy()
    # (a) the GPU pusher's samples, whole, through the oracle
    n_e = r0.shape[0]
    t = torch.empty(n_s + 1, dtype=torch.float64, device="cuda")
    out = [torch.empty((n_e, n_s + 1, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    lw.lw_boris_push(r.clone(), u.clone(), t0, (t1 - t0) / n_s, n_s, L, t, *out)
    torch.cuda.synchronize()
    S_a, st_a = _oracle_spectrum(t.cpu().numpy(), *(x.cpu().numpy() for x in out), n_hat, grid)
    assert st_a & ~oracle.ST_CLIP == 0
    tol = 1e-9 if precision == lw.LW_FP64 else 1e-4
    assert rel_l2(S_gpu, S_a) <= tol
    # (b) the numpy pusher's trajectories through the oracle
    ref = boris_trajectories(r0, u0, laser, t0, t1, n_s)
    S_b, _ = _oracle_spectrum(ref.t, ref.r, ref.beta, ref.beta_dot, n_hat, grid)
    tol_b = 1e-6 if precision == lw.LW_FP64 else 1e-4
    assert rel_l2(S_gpu, S_b) <= tol_b
