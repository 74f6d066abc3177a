"""Electron bunches pushed through a focused Gaussian laser pulse with the
Boris method (FP64, numpy, vectorised over electrons).

Laser: lowest-order paraxial Gaussian beam, polarised along x, propagating
along -z, focused at z = 0 and peaking there at t = 0:
    E_x = E0 (w0/w) exp(-rho^2/w^2) exp(-(t + z/c)^2/(2 sigma^2))
          * cos(omega (t + z/c) + k rho^2 zeta/(2 (zeta^2 + zR^2)) - atan(zeta/zR)),
    B_y = -E_x / c0,   zeta = -z,  w = w0 sqrt(1 + zeta^2/zR^2),  zR = pi w0^2 / lam,
with E0 = a0 m_e c0 omega / e and sigma = FWHM_intensity/(2 sqrt(ln 2)).

Pusher: drift-kick-drift with the Boris rotation (second order), positions
and momenta stored at the same uniform lab times; beta_dot at each sample is
the Lorentz-force derivative of beta at that sample's position and time:
    beta_dot = q/(m gamma c) [E + c beta x B - beta (beta . E)].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .physics import C0, M_E, Q_E
from .simple import Trajectories


@dataclass
class GaussianLaser:
    lam: float = 0.8e-6
    a0: float = 0.5
    w0: float = 20e-6
    fwhm: float = 30e-15

    @property
    def omega(self):
        return 2.0 * np.pi * C0 / self.lam

    @property
    def sigma(self):
        return self.fwhm / (2.0 * np.sqrt(np.log(2.0)))

    @property
    def E0(self):
        return self.a0 * M_E * C0 * self.omega / Q_E

    def fields(self, x, y, z, t):
        """(E, B) as arrays [..., 3] at positions (x, y, z) and time t."""
        k = self.omega / C0
        zR = np.pi * self.w0**2 / self.lam
        zeta = -z
        w = self.w0 * np.sqrt(1.0 + (zeta / zR) ** 2)
        rho2 = x * x + y * y
        xi = t + z / C0
        env = np.exp(-rho2 / (w * w)) * np.exp(-(xi * xi) / (2.0 * self.sigma**2))
        phase = (self.omega * xi + k * rho2 * zeta / (2.0 * (zeta * zeta + zR * zR))
                 - np.arctan(zeta / zR))
        Ex = self.E0 * (self.w0 / w) * env * np.cos(phase)
        zero = np.zeros_like(Ex)
        E = np.stack([Ex, zero, zero], axis=-1)
        B = np.stack([zero, -Ex / C0, zero], axis=-1)
        return E, B


def _lorentz_beta_dot(beta, gamma, E, B, qm):
    bxB = np.cross(beta, B)
    bE = np.sum(beta * E, axis=-1, keepdims=True)
    return (qm / (gamma[..., None] * C0)) * (E + C0 * bxB - beta * bE)


def boris_trajectories(r0, u0, laser: GaussianLaser, t_start: float, t_end: float,
                       n_steps: int, charge: float = -Q_E, mass: float = M_E,
                       out_dtype=np.float64) -> Trajectories:
    """Push electrons from (r0, u0 = gamma beta) at t_start to t_end in n_steps
    equal steps; returns samples at the n_steps+1 lab times."""
    r = np.array(r0, dtype=np.float64)
    u = np.array(u0, dtype=np.float64)
    n_e = r.shape[0]
    dt = (t_end - t_start) / n_steps
    t = t_start + dt * np.arange(n_steps + 1)
    qm = charge / mass
    R = np.empty((n_e, n_steps + 1, 3), dtype=out_dtype)
    BETA = np.empty_like(R)
    BD = np.empty_like(R)

    def record(i, r, u, ti):
        gam = np.sqrt(1.0 + np.sum(u * u, axis=-1))
        beta = u / gam[:, None]
        E, B = laser.fields(r[:, 0], r[:, 1], r[:, 2], ti)
        R[:, i] = r
        BETA[:, i] = beta
        BD[:, i] = _lorentz_beta_dot(beta, gam, E, B, qm)

    record(0, r, u, t[0])
    eps = qm * dt / (2.0 * C0)          # u is dimensionless: du/dt = (q/(m c)) (E + v x B)
    for i in range(n_steps):
        gam = np.sqrt(1.0 + np.sum(u * u, axis=-1))
        rh = r + (0.5 * dt * C0) * u / gam[:, None]
        E, B = laser.fields(rh[:, 0], rh[:, 1], rh[:, 2], t[i] + 0.5 * dt)
        um = u + eps * E
        gm = np.sqrt(1.0 + np.sum(um * um, axis=-1))
        tv = (qm * dt / (2.0 * gm))[:, None] * B
        up = um + np.cross(um, tv)
        s = 2.0 * tv / (1.0 + np.sum(tv * tv, axis=-1))[:, None]
        u = um + np.cross(up, s) + eps * E
        gam = np.sqrt(1.0 + np.sum(u * u, axis=-1))
        r = rh + (0.5 * dt * C0) * u / gam[:, None]
        record(i + 1, r, u, t[i + 1])
    return Trajectories(t, R, BETA, BD)


def gaussian_bunch(n_e: int, seed: int, sigma_x: float, sigma_y: float, sigma_z: float,
                   gamma_mean: float, gamma_rel_spread: float, eps_n: float,
                   t_start: float, cut: float = 4.0):
    """Sample a Gaussian bunch defined at t = 0 (centre at the origin, moving
    along +z) and drift it ballistically back to t_start.

    Angular spread sigma_x' = eps_n / (gamma sigma_x) (and likewise in y).
    Coordinates are drawn from a normal truncated at ``cut`` sigma.
    Returns (r0 [n_e][3], u0 [n_e][3]) at t_start.
    """
    rng = np.random.Generator(np.random.PCG64(seed))

    def tn(size):
        out = rng.normal(size=size)
        bad = np.abs(out) > cut
        while np.any(bad):
            out[bad] = rng.normal(size=int(bad.sum()))
            bad = np.abs(out) > cut
        return out

    x = tn(n_e) * sigma_x
    y = tn(n_e) * sigma_y
    z = tn(n_e) * sigma_z
    g = gamma_mean * (1.0 + gamma_rel_spread * tn(n_e))
    xp = tn(n_e) * (eps_n / (gamma_mean * sigma_x) if sigma_x > 0 else 0.0)
    yp = tn(n_e) * (eps_n / (gamma_mean * sigma_y) if sigma_y > 0 else 0.0)
    p = np.sqrt(g * g - 1.0)
    uz = p / np.sqrt(1.0 + xp * xp + yp * yp)
    u = np.stack([uz * xp, uz * yp, uz], axis=-1)
    v = C0 * u / g[:, None]
    r = np.stack([x, y, z], axis=-1) + v * t_start
    return r, u
