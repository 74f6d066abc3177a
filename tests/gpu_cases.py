"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded inputs."""
import numpy as np
import torch

import oracle
from paper_2206_03015_gb300 import lw


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def record_value(rec, precision):
    return lw.record_value(rec, precision).cpu().numpy()


def gpu_run(tr, n_hat, grid, precision, flags=lw.LW_FIELD_ACCEL, R=1.0, block=128,
            spectrum=True, want_X=False):
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot, block=block)
    det = lw.Detector(n_hat, R=R)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rec = lw.lw_deposit_time_domain(traj, det, grid, precision, flags, status=status)
    out = {"rec": record_value(rec, precision)}
    pow2 = grid.n_bins >= 2 and (grid.n_bins & (grid.n_bins - 1)) == 0
    if spectrum and pow2:
        res = lw.lw_spectrum(rec, precision, det.n_pix, grid, want_X=want_X)
        if want_X:
            out["S"], out["X"] = res[0].double().cpu().numpy(), res[1].cpu().numpy()
        else:
            out["S"] = res.double().cpu().numpy()
    torch.cuda.synchronize()
    out["status"] = int(status.item())
    return out


def gpu_bounds(tr, n_hat):
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot)
    b = lw.lw_grid_bounds(traj, lw.Detector(n_hat)).cpu().numpy()
    return float(b[0]), float(b[1])


def oracle_run(tr, n_hat, grid, flags=oracle.FLAG_ACCEL, R=1.0, spectrum=True, want_X=False):
    rec, st = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, grid.t_min, grid.dt_u,
                                 grid.n_bins, R=R, flags=flags)
    out = {"rec": rec, "status": st}
    if spectrum and grid.n_bins >= 2 and (grid.n_bins & (grid.n_bins - 1)) == 0:
        if want_X:
            out["S"], out["X"] = oracle.spectrum(rec, grid.dt_u, want_X=True)
        else:
            out["S"] = oracle.spectrum(rec, grid.dt_u)
    return out
