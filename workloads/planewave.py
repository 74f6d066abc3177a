"""Electron trajectories in a linearly polarised plane wave, from the analytic
light-front solution (head-on inverse Compton scattering).

The laser propagates along -z and is polarised along x; its normalised vector
potential depends only on the phase time xi = t + z/c0:
    a(xi) = a0 * exp(-xi^2 / (2 sigma^2)) * cos(omega_L xi),
with sigma = FWHM_intensity / (2 sqrt(ln 2)).  For an electron that enters
with gamma0 along +z the transverse canonical momentum and h = gamma + u_z are
conserved, so (u = gamma beta)
    u_x = a,  gamma = (h + (1 + a^2)/h)/2,  u_z = (h - (1 + a^2)/h)/2,
    dt/dxi = gamma/h,  dx/dxi = c0 a/h,  z = c0 (xi - t).
The time integral is done with 8-point Gauss-Legendre panels (about 64 panels
per carrier period) and inverted by Newton iteration at uniform lab times, so
the samples (t_i, r, beta, beta_dot) are consistent to ~1e-13 relative.
"""
from __future__ import annotations

import numpy as np

from .physics import C0
from .simple import Trajectories

_GL_X, _GL_W = np.polynomial.legendre.leggauss(8)


class _PlaneWave:
    def __init__(self, gamma0, lam, a0, fwhm):
        self.omega = 2.0 * np.pi * C0 / lam
        self.sigma = fwhm / (2.0 * np.sqrt(np.log(2.0)))
        self.a0 = a0
        self.gamma0 = gamma0
        self.h = gamma0 + np.sqrt(gamma0 * gamma0 - 1.0)

    def a(self, xi):
        return self.a0 * np.exp(-xi * xi / (2.0 * self.sigma**2)) * np.cos(self.omega * xi)

    def da(self, xi):
        g = self.a0 * np.exp(-xi * xi / (2.0 * self.sigma**2))
        return g * (-(xi / self.sigma**2) * np.cos(self.omega * xi)
                    - self.omega * np.sin(self.omega * xi))

    def gamma(self, xi):
        a = self.a(xi)
        return 0.5 * (self.h + (1.0 + a * a) / self.h)

    def dt_dxi(self, xi):
        return self.gamma(xi) / self.h

    def dx_dxi(self, xi):
        return C0 * self.a(xi) / self.h


class _Cumulative:
    """Cumulative integral F(xi) = int_{xi_lo}^{xi} f on a panel table."""

    def __init__(self, f, xi_lo, xi_hi, h):
        self.f = f
        self.lo = xi_lo
        self.h = h
        n = int(np.ceil((xi_hi - xi_lo) / h)) + 1
        edges = xi_lo + h * np.arange(n + 1)
        mid = 0.5 * (edges[:-1] + edges[1:])
        nodes = mid[:, None] + 0.5 * h * _GL_X[None, :]
        panel = 0.5 * h * (f(nodes) @ _GL_W)
        self.cum = np.concatenate([[0.0], np.cumsum(panel)])
        self.n = n

    def __call__(self, xi):
        xi = np.asarray(xi)
        p = np.clip(np.floor((xi - self.lo) / self.h).astype(np.int64), 0, self.n - 1)
        a = self.lo + self.h * p
        half = 0.5 * (xi - a)
        nodes = (a + half)[..., None] + half[..., None] * _GL_X
        part = half * (self.f(nodes) @ _GL_W)
        return self.cum[p] + part


def plane_wave_trajectories(gamma0: float, lam: float, a0: float, fwhm: float, t_start: float,
                            t_end: float, n_steps: int, n_e: int = 1, z_offsets=None,
                            x_offsets=None, y_offsets=None) -> Trajectories:
    """Sample n_e electrons at n_steps+1 uniform lab times in [t_start, t_end].

    Electron k is the light-front solution shifted so that, before the pulse,
    it sits z_offsets[k] further along +z than the reference electron (which
    is at z = 0 when the pulse peak passes z = 0 at t = 0); transverse offsets
    translate it rigidly (the plane wave is uniform in x and y).
    """
    pw = _PlaneWave(gamma0, lam, a0, fwhm)
    beta0 = np.sqrt(1.0 - 1.0 / gamma0**2)
    zo = np.zeros(n_e) if z_offsets is None else np.asarray(z_offsets, dtype=np.float64)
    xo = np.zeros(n_e) if x_offsets is None else np.asarray(x_offsets, dtype=np.float64)
    yo = np.zeros(n_e) if y_offsets is None else np.asarray(y_offsets, dtype=np.float64)
    # a pure spatial offset dz before the pulse = lab-time shift of the
    # light-front solution by Delta = -dz / (c0 (1 + beta0))
    shift = -zo / (C0 * (1.0 + beta0))
    t = t_start + (t_end - t_start) * np.arange(n_steps + 1) / n_steps
    xi_lo = 2.0 * (t_start - np.max(shift)) - 4.0 * np.max(np.abs(zo)) / C0 - 1e-15
    xi_hi = 2.0 * (t_end - np.min(shift)) + 4.0 * np.max(np.abs(zo)) / C0 + 1e-15
    h = 2.0 * np.pi / pw.omega / 64.0
    T_of = _Cumulative(pw.dt_dxi, xi_lo, xi_hi, h)
    X_of = _Cumulative(pw.dx_dxi, xi_lo, xi_hi, h)
    T0 = T_of(np.array(0.0))
    X0 = X_of(np.array(0.0))
    tgt = t[None, :] - shift[:, None]                   # base-solution time
    xi = 2.0 * tgt
    for _ in range(8):
        f = T_of(xi) - T0 - tgt
        xi = xi - f / pw.dt_dxi(xi)
    tk = T_of(xi) - T0 + shift[:, None]
    a = pw.a(xi)
    da = pw.da(xi)
    gam = pw.gamma(xi)
    uz = 0.5 * (pw.h - (1.0 + a * a) / pw.h)
    x = X_of(xi) - X0 + xo[:, None]
    z = C0 * (xi - tk)
    r = np.stack([x, np.broadcast_to(yo[:, None], x.shape), z], axis=-1)
    beta = np.stack([a / gam, np.zeros_like(a), uz / gam], axis=-1)
    bdx = (da * pw.h / gam**2) * (1.0 - a * a / (pw.h * gam))
    bdz = -a * da * pw.h / gam**3
    bd = np.stack([bdx, np.zeros_like(a), bdz], axis=-1)
    return Trajectories(np.ascontiguousarray(t), np.ascontiguousarray(r),
                        np.ascontiguousarray(beta), np.ascontiguousarray(bd))


def doppler_fundamental(gamma0: float, lam: float, a0: float, theta: float = 0.0) -> float:
    """Textbook on-axis ICS line omega_1 = 4 gamma^2 omega_L / (1 + a0^2/2 + gamma^2 theta^2)."""
    omega_l = 2.0 * np.pi * C0 / lam
    return 4.0 * gamma0**2 * omega_l / (1.0 + 0.5 * a0**2 + gamma0**2 * theta**2)
