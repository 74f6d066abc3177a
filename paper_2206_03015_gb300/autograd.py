"""Differentiable spectra: gradients of a band-integrated spectral yield with
respect to per-electron initial momenta and the laser's a0 and waist.

``PushSpectrum`` is the whole chain in the library's kernels: the GPU Boris push
(lw_boris_push), the FP64 deposit and spectrum, and in reverse lw_spectrum_grad
followed by lw_boris_push_grad (the push differentiated in forward mode along
u0, a0 and w0, so no trajectory state is stored or recomputed).

``LWSpectrum`` wraps the library's FP64 forward (upload, deposit, spectrum)
and its adjoint (lw_spectrum_grad) as a torch.autograd.Function of the
trajectory samples (r, beta, beta_dot).  ``boris_push`` produces those samples
from initial conditions and laser parameters with the Boris method written in
torch, so autograd carries the gradient on to (u0, a0, w0); the pusher is
split into segments of ``checkpoint_every`` steps that are recomputed during
the backward pass, so the autograd graph holds one segment at a time.  It is
the independent formulation the kernel chain is tested against.
"""
from __future__ import annotations

import math

import torch
from torch.utils.checkpoint import checkpoint

from . import lw

C0 = 299792458.0
Q_E = 1.602176634e-19
M_E = 9.1093837015e-31


def _sections(precision):
    """Trajectory sections a forward in `precision` and its adjoint read (the adjoint
    always reads the FP64 samples)."""
    if precision == lw.LW_FP64:
        return lw.LW_SECTION_FP64
    return lw.LW_SECTION_FP64 | lw.LW_SECTION_MIXED


class LWSpectrum(torch.autograd.Function):
    """S[m][l] of trajectories (t, r, beta, beta_dot) for a detector and grid: FP64 with
    `precision` LW_FP64 (the default), FP32 with a mixed mode (mixed deposit and spectrum,
    mixed-precision adjoint)."""

    @staticmethod
    def forward(ctx, t, r, beta, beta_dot, det: "lw.Detector", grid: "lw.Grid", q: float = Q_E,
                precision: int = lw.LW_FP64):
        traj = lw.lw_trajectories_upload(t.detach(), r.detach(), beta.detach(),
                                         beta_dot.detach(), sections=_sections(precision),
                                         device=det.n_hat.device)
        rec = lw.lw_deposit_time_domain(traj, det, grid, precision)
        S, X = lw.lw_spectrum(rec, precision, det.n_pix, grid, q=q, want_X=True)
        ctx.traj, ctx.det, ctx.grid, ctx.q, ctx.precision = traj, det, grid, q, precision
        ctx.save_for_backward(X)
        return S

    @staticmethod
    def backward(ctx, gS):
        (X,) = ctx.saved_tensors
        g_r, g_b, g_a = lw.lw_spectrum_grad(ctx.traj, ctx.det, ctx.grid, X, gS.contiguous(),
                                            q=ctx.q, precision=ctx.precision)
        return None, g_r, g_b, g_a, None, None, None, None


class PushSpectrum(torch.autograd.Function):
    """S[m][l] of electrons pushed by the library's Boris kernel (lw_boris_push) from
    (r0, u0) through the Gaussian laser (lam, a0, w0, fwhm), as a function of u0 [n_e, 3] and
    the 0-d tensors a0 and w0; FP64 with `precision` LW_FP64, FP32 with a mixed mode.
    Backward: lw_spectrum_grad (deposit and FFT transposed, in the forward's precision) then
    lw_boris_push_grad (the push differentiated in forward mode along u0, a0 and w0) -- every
    step in the library's kernels."""

    @staticmethod
    def forward(ctx, u0, a0, w0, r0, lam: float, fwhm: float, t_start: float, t_end: float,
                n_steps: int, det: "lw.Detector", grid: "lw.Grid", q: float = Q_E,
                precision: int = lw.LW_FP64):
        dev = u0.device
        n_e = u0.shape[0]
        dt = (t_end - t_start) / n_steps
        laser = (lam, float(a0), float(w0), fwhm)
        t = torch.empty(n_steps + 1, dtype=torch.float64, device=dev)
        R, B, A = (torch.empty((n_e, n_steps + 1, 3), dtype=torch.float64, device=dev)
                   for _ in range(3))
        r0 = r0.detach().to(torch.float64).contiguous()
        u0d = u0.detach().to(torch.float64).contiguous()
        lw.lw_boris_push(r0.clone(), u0d.clone(), t_start, dt, n_steps, laser, t, R, B, A)
        traj = lw.lw_trajectories_upload(t, R, B, A, sections=_sections(precision), device=dev)
        rec = lw.lw_deposit_time_domain(traj, det, grid, precision)
        S, X = lw.lw_spectrum(rec, precision, det.n_pix, grid, q=q, want_X=True)
        ctx.traj, ctx.det, ctx.grid, ctx.q, ctx.precision = traj, det, grid, q, precision
        ctx.push = (t_start, dt, n_steps, laser)
        ctx.save_for_backward(X, r0, u0d)
        return S

    @staticmethod
    def backward(ctx, gS):
        X, r0, u0 = ctx.saved_tensors
        g_r, g_b, g_a = lw.lw_spectrum_grad(ctx.traj, ctx.det, ctx.grid, X, gS.contiguous(),
                                            q=ctx.q, precision=ctx.precision)
        t_start, dt, n_steps, laser = ctx.push
        du0, dlaser = lw.lw_boris_push_grad(r0, u0, t_start, dt, n_steps, laser, g_r, g_b, g_a)
        return (du0, dlaser[0], dlaser[1], None, None, None, None, None, None, None, None, None,
                None)


def band_mask(grid: "lw.Grid", omega_center: float, rel_half_width: float = 0.05):
    """1 on |omega_l - omega_c| <= rel_half_width * omega_c, else 0 (float64)."""
    om = grid.omega
    return ((om - omega_center).abs() <= rel_half_width * omega_center).to(torch.float64)


def band_energy(S, grid: "lw.Grid", mask):
    """sum over pixels and the band of S d_omega (J / sr summed over pixels)."""
    d_omega = 2.0 * math.pi / (grid.n_bins * grid.dt_u)
    return (S * mask.to(S.device)[None, :]).sum() * d_omega


def _laser_fields(x, y, z, t, a0, w0, lam, fwhm):
    """Lowest-order paraxial Gaussian beam along -z, polarised x (as in the workloads)."""
    omega = 2.0 * math.pi * C0 / lam
    k = omega / C0
    sigma = fwhm / (2.0 * math.sqrt(math.log(2.0)))
    E0 = a0 * M_E * C0 * omega / Q_E
    zR = math.pi * w0 * w0 / lam
    zeta = -z
    w = w0 * torch.sqrt(1.0 + (zeta / zR) ** 2)
    rho2 = x * x + y * y
    xi = t + z / C0
    env = torch.exp(-rho2 / (w * w)) * torch.exp(-(xi * xi) / (2.0 * sigma * sigma))
    phase = omega * xi + k * rho2 * zeta / (2.0 * (zeta * zeta + zR * zR)) - torch.atan(zeta / zR)
    Ex = E0 * (w0 / w) * env * torch.cos(phase)
    zero = torch.zeros_like(Ex)
    return torch.stack([Ex, zero, zero], -1), torch.stack([zero, -Ex / C0, zero], -1)


def _beta_dot(beta, gam, E, B, qm):
    bxB = torch.cross(beta, B, dim=-1)
    bE = (beta * E).sum(-1, keepdim=True)
    return (qm / (gam[..., None] * C0)) * (E + C0 * bxB - beta * bE)


def _sample(r, u, t, a0, w0, lam, fwhm, qm):
    gam = torch.sqrt(1.0 + (u * u).sum(-1))
    beta = u / gam[:, None]
    E, B = _laser_fields(r[:, 0], r[:, 1], r[:, 2], t, a0, w0, lam, fwhm)
    return beta, _beta_dot(beta, gam, E, B, qm)


def _segment(r, u, a0, w0, t0, dt, n, lam, fwhm, qm):
    """n drift-kick-drift Boris steps from time t0; returns the samples after each step."""
    eps = qm * dt / (2.0 * C0)
    Rs, Bs, As = [], [], []
    for s in range(n):
        ti = t0 + s * dt
        gam = torch.sqrt(1.0 + (u * u).sum(-1))
        rh = r + (0.5 * dt * C0) * u / gam[:, None]
        E, B = _laser_fields(rh[:, 0], rh[:, 1], rh[:, 2], ti + 0.5 * dt, a0, w0, lam, fwhm)
        um = u + eps * E
        gm = torch.sqrt(1.0 + (um * um).sum(-1))
        tv = (qm * dt / (2.0 * gm))[:, None] * B
        up = um + torch.cross(um, tv, dim=-1)
        sv = 2.0 * tv / (1.0 + (tv * tv).sum(-1))[:, None]
        u = um + torch.cross(up, sv, dim=-1) + eps * E
        gam = torch.sqrt(1.0 + (u * u).sum(-1))
        r = rh + (0.5 * dt * C0) * u / gam[:, None]
        b, a = _sample(r, u, ti + dt, a0, w0, lam, fwhm, qm)
        Rs.append(r)
        Bs.append(b)
        As.append(a)
    return torch.stack(Rs, 1), torch.stack(Bs, 1), torch.stack(As, 1), r, u


def boris_push(r0, u0, a0, w0, lam: float, fwhm: float, t_start: float, t_end: float,
               n_steps: int, checkpoint_every: int = 256, charge: float = -Q_E,
               mass: float = M_E):
    """Differentiable Boris push (FP64).  r0, u0: [n_e, 3] tensors (u = gamma beta);
    a0, w0: 0-d tensors.  Returns (t [n_s+1], r, beta, beta_dot [n_e, n_s+1, 3])."""
    qm = charge / mass
    dt = (t_end - t_start) / n_steps
    t = t_start + dt * torch.arange(n_steps + 1, dtype=torch.float64, device=r0.device)
    b0, bd0 = _sample(r0, u0, t_start, a0, w0, lam, fwhm, qm)
    Rs, Bs, As = [r0[:, None]], [b0[:, None]], [bd0[:, None]]
    r, u = r0, u0
    for s0 in range(0, n_steps, checkpoint_every):
        n = min(checkpoint_every, n_steps - s0)
        fn = (lambda r_, u_, a_, w_, s0=s0, n=n:
              _segment(r_, u_, a_, w_, t_start + s0 * dt, dt, n, lam, fwhm, qm))
        R, B, A, r, u = checkpoint(fn, r, u, a0, w0, use_reentrant=False)
        Rs.append(R)
        Bs.append(B)
        As.append(A)
    return t, torch.cat(Rs, 1), torch.cat(Bs, 1), torch.cat(As, 1)
