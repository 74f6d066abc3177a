"""Small synthetic trajectories with known structure, for pins and edge cases."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .physics import C0


@dataclass
class Trajectories:
    """t [n_s+1] (shared) or [n_e][n_s+1]; r, beta, beta_dot [n_e][n_s+1][3] (float64)."""
    t: np.ndarray
    r: np.ndarray
    beta: np.ndarray
    beta_dot: np.ndarray

    @property
    def n_e(self) -> int:
        return self.r.shape[0]

    @property
    def n_s(self) -> int:
        return self.r.shape[1] - 1

    def subset(self, idx) -> "Trajectories":
        t = self.t if self.t.ndim == 1 else self.t[idx]
        return Trajectories(t, self.r[idx], self.beta[idx], self.beta_dot[idx])

    def concat(self, other: "Trajectories") -> "Trajectories":
        assert self.t.ndim == 1 and np.array_equal(self.t, other.t)
        return Trajectories(self.t, np.concatenate([self.r, other.r]),
                            np.concatenate([self.beta, other.beta]),
                            np.concatenate([self.beta_dot, other.beta_dot]))


def stationary_constant_acceleration(n_s: int, dt: float, accel, n_e: int = 1,
                                     t0: float = 0.0) -> Trajectories:
    """A charge at rest at the origin with constant beta_dot (beta stays 0)."""
    t = t0 + dt * np.arange(n_s + 1)
    r = np.zeros((n_e, n_s + 1, 3))
    beta = np.zeros_like(r)
    bd = np.broadcast_to(np.asarray(accel, dtype=np.float64), r.shape).copy()
    return Trajectories(t, r, beta, bd)


def linear_ramp_acceleration(n_s: int, dt: float, a0, a1, n_e: int = 1,
                             t0: float = 0.0) -> Trajectories:
    """At rest at the origin, beta_dot = a0 + a1 * (t - t0) (linear in time)."""
    t = t0 + dt * np.arange(n_s + 1)
    r = np.zeros((n_e, n_s + 1, 3))
    beta = np.zeros_like(r)
    a0 = np.asarray(a0, dtype=np.float64)
    a1 = np.asarray(a1, dtype=np.float64)
    bd = a0[None, None, :] + a1[None, None, :] * (t - t0)[None, :, None]
    bd = np.broadcast_to(bd, r.shape).copy()
    return Trajectories(t, r, beta, bd)


def uniform_motion(n_s: int, dt: float, beta_vec, r0=(0.0, 0.0, 0.0), t0: float = 0.0,
                   n_e: int = 1) -> Trajectories:
    """Uniform straight-line motion r = r0 + c beta (t - 0), beta_dot = 0."""
    t = t0 + dt * np.arange(n_s + 1)
    b = np.asarray(beta_vec, dtype=np.float64)
    r = np.asarray(r0, dtype=np.float64)[None, :] + C0 * b[None, :] * t[:, None]
    r = np.broadcast_to(r, (n_e, n_s + 1, 3)).copy()
    beta = np.broadcast_to(b, r.shape).copy()
    return Trajectories(t, r, beta, np.zeros_like(r))


def circular_motion(n_s: int, dt: float, beta0: float, omega: float, n_e: int = 1,
                    phase0: float = 0.0) -> Trajectories:
    """Circular orbit in the x-y plane with speed beta0 c and angular frequency omega."""
    t = dt * np.arange(n_s + 1)
    ph = phase0 + omega * t
    rad = beta0 * C0 / omega
    r = np.stack([rad * np.cos(ph), rad * np.sin(ph), np.zeros_like(ph)], axis=-1)
    beta = np.stack([-beta0 * np.sin(ph), beta0 * np.cos(ph), np.zeros_like(ph)], axis=-1)
    bd = np.stack([-beta0 * omega * np.cos(ph), -beta0 * omega * np.sin(ph),
                   np.zeros_like(ph)], axis=-1)
    rep = lambda a: np.broadcast_to(a, (n_e,) + a.shape).copy()  # noqa: E731
    return Trajectories(t, rep(r), rep(beta), rep(bd))


def random_smooth(n_e: int, n_s: int, dt: float, seed: int, gamma: float = 20.0,
                  amp: float = 0.02, n_modes: int = 3, t_per_electron: bool = False,
                  spread: float = 2e-7) -> Trajectories:
    """Electrons moving mostly along +z with a smooth random transverse wiggle.

    beta_perp(t) = sum of a few random sinusoids (amplitude ~amp/gamma); beta_z
    follows from a fixed gamma; r is the exact integral of c beta, beta_dot the
    exact derivative, so the record is a genuine, physically consistent input.
    Initial positions are spread by ``spread`` metres in x, y and z.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t_base = dt * np.arange(n_s + 1)
    if t_per_electron:
        offs = rng.uniform(-0.3, 0.3, size=(n_e, 1)) * dt * n_s
        t = t_base[None, :] + offs
    else:
        t = t_base
    tt = np.broadcast_to(t if t.ndim == 2 else t[None, :], (n_e, n_s + 1))
    T = dt * n_s
    w = rng.uniform(2.0, 9.0, size=(n_e, 2, n_modes)) * (2 * np.pi / T)
    a = rng.normal(size=(n_e, 2, n_modes)) * (amp / gamma / np.sqrt(n_modes))
    ph = rng.uniform(0, 2 * np.pi, size=(n_e, 2, n_modes))
    arg = w[:, :, :, None] * tt[:, None, None, :] + ph[:, :, :, None]
    bperp = np.sum(a[..., None] * np.sin(arg), axis=2)            # [n_e,2,ns+1]
    bperp_dot = np.sum((a * w)[..., None] * np.cos(arg), axis=2)
    xperp = np.sum((-a / w)[..., None] * np.cos(arg), axis=2) * C0
    b_tot2 = 1.0 - 1.0 / gamma**2
    bz = np.sqrt(b_tot2 - bperp[:, 0] ** 2 - bperp[:, 1] ** 2)
    bz_dot = -(bperp[:, 0] * bperp_dot[:, 0] + bperp[:, 1] * bperp_dot[:, 1]) / bz
    # z = integral of c*bz dt by composite Simpson on a refined grid per sample
    r0 = rng.normal(size=(n_e, 3)) * spread
    z = np.empty((n_e, n_s + 1))
    z[:, 0] = 0.0
    sub = 8
    for i in range(n_s):
        ta = tt[:, i][:, None] + (tt[:, i + 1] - tt[:, i])[:, None] * np.linspace(0, 1, sub + 1)
        argr = w[:, :, :, None] * ta[:, None, None, :] + ph[:, :, :, None]
        bp = np.sum(a[..., None] * np.sin(argr), axis=2)
        bzz = np.sqrt(b_tot2 - bp[:, 0] ** 2 - bp[:, 1] ** 2)
        h = (tt[:, i + 1] - tt[:, i]) / sub
        wts = np.ones(sub + 1)
        wts[1:-1:2] = 4
        wts[2:-1:2] = 2
        z[:, i + 1] = z[:, i] + C0 * h / 3.0 * (bzz @ wts)
    z = z + C0 * 0.0
    r = np.stack([xperp[:, 0] + r0[:, 0:1], xperp[:, 1] + r0[:, 1:2], z + r0[:, 2:3]], axis=-1)
    beta = np.stack([bperp[:, 0], bperp[:, 1], bz], axis=-1)
    bd = np.stack([bperp_dot[:, 0], bperp_dot[:, 1], bz_dot], axis=-1)
    return Trajectories(np.ascontiguousarray(t), np.ascontiguousarray(r),
                        np.ascontiguousarray(beta), np.ascontiguousarray(bd))


def transverse_oscillation(n_e: int, n_s: int, dt: float, beta_z: float, amp: float,
                           samples_per_period: float, seed: int = 0) -> Trajectories:
    """Electrons drifting along z at beta_z with a transverse velocity oscillation
    beta_x = amp sin(omega t + phase_k), sampled samples_per_period times per period
    (positions integrated analytically, beta_dot = d beta / dt).  Few samples per period
    make the field change by a large fraction across each step."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = dt * np.arange(n_s + 1, dtype=np.float64)
    omega = 2.0 * np.pi / (samples_per_period * dt)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=(n_e, 1))
    z0 = rng.normal(scale=1e-9, size=(n_e, 1))
    r = np.zeros((n_e, n_s + 1, 3))
    beta = np.zeros_like(r)
    bd = np.zeros_like(r)
    r[..., 0] = -amp * C0 / omega * np.cos(omega * t + ph)
    r[..., 2] = z0 + beta_z * C0 * t
    beta[..., 0] = amp * np.sin(omega * t + ph)
    beta[..., 2] = beta_z
    bd[..., 0] = amp * omega * np.cos(omega * t + ph)
    return Trajectories(t, r, beta, bd)
