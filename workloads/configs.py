"""Named synthetic workloads shaped like the paper's inverse Compton
scattering cases.  Seeds are PCG64(20603015 + id).  Every field needed to
rebuild a workload is stored on the returned object, so the oracle and the
CUDA library receive identical bytes.

  c1_tiny      16 electrons, gamma = 50 exactly, zero emittance, on axis, head-on with a
               linearly polarised plane wave (lambda = 1 um, a0 = 0.1, intensity FWHM
               10 fs); analytic trajectories at 2,000 uniform lab steps; 32x32 pixels
               spanning +-1/gamma; 4,096 observer bins.
  c1_offsets   as c1_tiny with electron k displaced by k*1 nm along z.
  c2_paper     10,000 electrons, Gaussian bunch sigma_x = sigma_y = 5 um, sigma_z = 10 um,
               gamma 60 with 0.1% rms spread, eps_n = 0.5 mm mrad; laser lambda = 0.8 um,
               a0 = 0.5, w0 = 20 um, FWHM 30 fs; Boris, 10,000 steps; 64x64 pixels over
               +-1.5/gamma; 65,536 bins.
  c2x          Nyquist-resolved variant of c2_paper (sigma_z = 0.1 um,
               sigma_x = sigma_y = 0.5 um, 64 electrons, 16x16 pixels).
  c4_grad      2,048 co-located on-axis electrons, gamma ~ N(60, 0.1%), Gaussian laser
               lambda = 1 um, a0 = 1.0, w0 = 20 um, FWHM 10 fs; 4,096 steps; 32x32 pixels;
               16,384 bins.
Any workload can be scaled down (``n_e``, ``n_s``, pixels, bins) for tests.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .boris import GaussianLaser, gaussian_bunch
from .parallel import boris_trajectories_parallel
from .detector import detector_grid
from .physics import C0, Q_E
from .planewave import plane_wave_trajectories
from .simple import Trajectories

SEED_BASE = 20603015


@dataclass
class Workload:
    name: str
    traj: Trajectories
    n_hat: np.ndarray
    n_bins: int
    R: float = 1.0
    q: float = Q_E
    gamma: float = 1.0
    lam: float = 1e-6
    a0: float = 0.0
    theta_x: np.ndarray | None = None
    theta_y: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_pix(self):
        return self.n_hat.shape[0]

    @property
    def deposits(self):
        """electron * step * pixel triples (the paper's N_p N_s N_obs)."""
        return self.traj.n_e * self.traj.n_s * self.n_pix


def c1_tiny(n_e=16, n_s=2000, nx=32, n_bins=4096, z_offset_step=0.0) -> Workload:
    gamma, lam, a0, fwhm = 50.0, 1e-6, 0.1, 10e-15
    sigma = fwhm / (2.0 * np.sqrt(np.log(2.0)))
    t_half = 0.5 * sigma * np.sqrt(2.0 * np.log(1e6))      # envelope 1e-6 at both ends
    zo = z_offset_step * np.arange(n_e)
    tr = plane_wave_trajectories(gamma, lam, a0, fwhm, -t_half, t_half, n_s, n_e=n_e,
                                 z_offsets=zo)
    n_hat, tx, ty = detector_grid(nx, nx, 1.0 / gamma)
    return Workload("c1_tiny" if z_offset_step == 0 else "c1_offsets", tr, n_hat, n_bins,
                    gamma=gamma, lam=lam, a0=a0, theta_x=tx, theta_y=ty,
                    meta=dict(fwhm=fwhm, t_half=t_half))


def c1_offsets(**kw) -> Workload:
    kw.setdefault("z_offset_step", 1e-9)
    return c1_tiny(**kw)


def _c2_like(name, n_e, n_s, nx, n_bins, sigma_x, sigma_y, sigma_z, seed, half_angle_g=1.5,
             t_half=None, laser=None, gamma=60.0, spread=1e-3, eps_n=0.5e-6):
    laser = laser or GaussianLaser(lam=0.8e-6, a0=0.5, w0=20e-6, fwhm=30e-15)
    if t_half is None:
        env = laser.sigma * np.sqrt(2.0 * np.log(1e6))
        t_half = 0.5 * (env + 4.0 * sigma_z / C0) * 1.05
    r0, u0 = gaussian_bunch(n_e, seed, sigma_x, sigma_y, sigma_z, gamma, spread, eps_n, -t_half)
    tr = boris_trajectories_parallel(r0, u0, laser, -t_half, t_half, n_s)
    n_hat, tx, ty = detector_grid(nx, nx, half_angle_g / gamma)
    return Workload(name, tr, n_hat, n_bins, gamma=gamma, lam=laser.lam, a0=laser.a0,
                    theta_x=tx, theta_y=ty,
                    meta=dict(t_half=t_half, laser=laser, sigma=(sigma_x, sigma_y, sigma_z)))


def c2_paper(n_e=10_000, n_s=10_000, nx=64, n_bins=65_536) -> Workload:
    return _c2_like("c2_paper", n_e, n_s, nx, n_bins, 5e-6, 5e-6, 10e-6, SEED_BASE + 2)


def c2x(n_e=64, n_s=4000, nx=16, n_bins=1 << 15) -> Workload:
    return _c2_like("c2x", n_e, n_s, nx, n_bins, 0.5e-6, 0.5e-6, 0.1e-6, SEED_BASE + 6)


def c4_grad(n_e=2048, n_s=4096, nx=32, n_bins=16_384) -> Workload:
    laser = GaussianLaser(lam=1e-6, a0=1.0, w0=20e-6, fwhm=10e-15)
    return _c2_like("c4_grad", n_e, n_s, nx, n_bins, 0.0, 0.0, 0.0, SEED_BASE + 4,
                    half_angle_g=1.0, laser=laser, eps_n=0.0)


def c4_setup(n_e=2048, n_s=4096, nx=32, n_bins=16_384):
    """Initial state of config 4 without pushing it: (r0, u0, laser, t_start, t_end, n_s,
    n_hat, n_bins, gamma) -- the same bunch and laser as c4_grad."""
    laser = GaussianLaser(lam=1e-6, a0=1.0, w0=20e-6, fwhm=10e-15)
    gamma = 60.0
    env = laser.sigma * np.sqrt(2.0 * np.log(1e6))
    t_half = 0.5 * env * 1.05
    r0, u0 = gaussian_bunch(n_e, SEED_BASE + 4, 0.0, 0.0, 0.0, gamma, 1e-3, 0.0, -t_half)
    n_hat, _, _ = detector_grid(nx, nx, 1.0 / gamma)
    return r0, u0, laser, -t_half, t_half, n_s, n_hat, n_bins, gamma


def c5_batch(n_variants=64, seed=SEED_BASE + 5, n_e=(512, 8192), n_s=(2000, 40000),
             nx=(16, 128), log2_bins=(12, 17), gamma=(20.0, 200.0), a0=(0.05, 1.0)):
    """Batched design sweep: independent variants with gamma log-uniform, a0 uniform,
    electrons / steps / detector side log-uniform and 2^U{log2_bins} observer bins;
    each variant is a Gaussian bunch (as c2_paper) in a 0.8 um Gaussian laser.
    The default ranges are the full sweep; tests and benches pass smaller ranges.
    Returns a list of Workloads (trajectories generated lazily by ``.build()``)."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def logu(lo, hi, size):
        return np.exp(rng.uniform(np.log(lo), np.log(hi), size))

    g = logu(gamma[0], gamma[1], n_variants)
    a = rng.uniform(a0[0], a0[1], n_variants)
    ne = np.round(logu(n_e[0], n_e[1], n_variants)).astype(int)
    ns = np.round(logu(n_s[0], n_s[1], n_variants)).astype(int)
    side = np.round(logu(nx[0], nx[1], n_variants)).astype(int)
    lb = rng.integers(log2_bins[0], log2_bins[1] + 1, n_variants)
    out = []
    for v in range(n_variants):
        laser = GaussianLaser(lam=0.8e-6, a0=float(a[v]), w0=20e-6, fwhm=30e-15)
        out.append(_LazyVariant(f"c5_v{v}", int(ne[v]), int(ns[v]), int(side[v]), 1 << int(lb[v]),
                                float(g[v]), laser, seed + 1000 + v))
    return out


@dataclass
class _LazyVariant:
    name: str
    n_e: int
    n_s: int
    nx: int
    n_bins: int
    gamma: float
    laser: GaussianLaser
    seed: int

    @property
    def deposits(self):
        return self.n_e * self.n_s * self.nx * self.nx

    def build(self) -> Workload:
        return _c2_like(self.name, self.n_e, self.n_s, self.nx, self.n_bins, 5e-6, 5e-6, 10e-6,
                        self.seed, laser=self.laser, gamma=self.gamma)

    def initial_state(self):
        """What build() pushes, without pushing it: (r0, u0, t_start, t_end, n_hat) -- the
        same bunch, time window and detector, for a pusher of the caller's choice."""
        env = self.laser.sigma * np.sqrt(2.0 * np.log(1e6))
        t_half = 0.5 * (env + 4.0 * 10e-6 / C0) * 1.05
        r0, u0 = gaussian_bunch(self.n_e, self.seed, 5e-6, 5e-6, 10e-6, self.gamma, 1e-3,
                                0.5e-6, -t_half)
        n_hat, _, _ = detector_grid(self.nx, self.nx, 1.5 / self.gamma)
        return r0, u0, -t_half, t_half, n_hat
