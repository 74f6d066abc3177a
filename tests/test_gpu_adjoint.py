"""Adjoint (lw_spectrum_grad, FP64 and mixed precision) against central finite differences
of the CPU oracle and against the oracle's own gradient, and the end-to-end gradient
of a band-integrated spectral yield with respect to initial momenta and the
laser a0 / waist (differentiable
Boris pusher + LWSpectrum) against finite differences of the oracle fed by
the workload generator's pusher.  Tolerance 1e-3 relative.

The loss is continuous but its slope jumps whenever a sample's advanced time
crosses a grid point (Algorithm 2's interval of grid points changes), so a
central difference whose stencil straddles such a crossing does not measure
the derivative.  The end-to-end check therefore takes, per input, the largest
of a few steps (1e-7 ... 3e-9 relative) for which the plus and minus
trajectories give every sample the same grid interval in every direction, and
compares the adjoint with that kink-free difference quotient."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2206_03015_gb300 import lw
from paper_2206_03015_gb300.autograd import (LWSpectrum, PushSpectrum, band_energy, band_mask,
                                             boris_push)
from workloads import simple
from workloads.boris import GaussianLaser, boris_trajectories
from workloads.planewave import doppler_fundamental

pytestmark = pytest.mark.gpu
TOL = 1e-3


def _dirs(n, seed, max_angle):
    rng = np.random.Generator(np.random.PCG64(seed))
    tx = rng.uniform(-max_angle, max_angle, n)
    ty = rng.uniform(-max_angle, max_angle, n)
    return np.stack([np.sin(tx), np.cos(tx) * np.sin(ty), np.cos(tx) * np.cos(ty)], -1)


def _oracle_loss(tr, n_hat, grid, w):
    rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, grid.t_min, grid.dt_u,
                                grid.n_bins)
    return float(np.sum(w * oracle.spectrum(rec, grid.dt_u)))


def test_spectrum_grad_matches_oracle_finite_differences():
    tr = simple.random_smooth(3, 60, 2e-18, 301, gamma=5.0, amp=0.5)
    n_hat = _dirs(6, 7, 0.3)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    grid = lw.Grid(lo - 3 * (hi - lo) / 256, (hi - lo) / 250, 256)
    rng = np.random.Generator(np.random.PCG64(9))
    w = rng.uniform(0.5, 1.5, size=(6, 129))
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot, sections=lw.LW_SECTION_FP64)
    det = lw.Detector(n_hat)
    rec = lw.lw_deposit_time_domain(traj, det, grid, lw.LW_FP64)
    S, X = lw.lw_spectrum(rec, lw.LW_FP64, det.n_pix, grid, want_X=True)
    g = lw.lw_spectrum_grad(traj, det, grid, X, torch.from_numpy(w).cuda())
    grads = [x.cpu().numpy() for x in g]
    torch.cuda.synchronize()
    names = ("r", "beta", "beta_dot")
    checked = 0
    for which, arr in enumerate((tr.r, tr.beta, tr.beta_dot)):
        scale = np.abs(arr).max()
        for (k, i, c) in ((0, 17, 0), (1, 30, 2), (2, 44, 1), (0, 52, 2)):
            h = 1e-6 * scale
            plus = [a.copy() for a in (tr.r, tr.beta, tr.beta_dot)]
            minus = [a.copy() for a in (tr.r, tr.beta, tr.beta_dot)]
            plus[which][k, i, c] += h
            minus[which][k, i, c] -= h
            Lp = _oracle_loss(simple.Trajectories(tr.t, *plus), n_hat, grid, w)
            Lm = _oracle_loss(simple.Trajectories(tr.t, *minus), n_hat, grid, w)
            fd = (Lp - Lm) / (2 * h)
            ref = max(abs(fd), 1e-3 * np.abs(grads[which]).max())
            assert abs(grads[which][k, i, c] - fd) <= TOL * ref, (names[which], k, i, c,
                                                                  grads[which][k, i, c], fd)
            checked += 1
    assert checked == 12


@pytest.mark.parametrize("t_per_electron", [False, True])
def test_spectrum_grad_matches_oracle_gradient(t_per_electron):
    """lw_spectrum_grad against the oracle's own gradient (the chain rule written out in
    plain C, pinned by central differences of the oracle's loss), element by element: both
    FP64 with the same interval decisions, so they agree to rounding (1e-9 of the largest
    element)."""
    tr = simple.random_smooth(4, 90, 2e-18, 41, gamma=6.0, amp=0.4,
                              t_per_electron=t_per_electron)
    n_hat = _dirs(7, 5, 0.25)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    grid = lw.Grid(lo - 2.5 * (hi - lo) / 500, (hi - lo) / 500, 512)
    rng = np.random.Generator(np.random.PCG64(17))
    w = rng.uniform(0.2, 2.0, size=(7, 257))
    ref = oracle.tdm_grad(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, grid.t_min, grid.dt_u,
                          grid.n_bins, w)
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot, sections=lw.LW_SECTION_FP64)
    det = lw.Detector(n_hat)
    rec = lw.lw_deposit_time_domain(traj, det, grid, lw.LW_FP64)
    S, X = lw.lw_spectrum(rec, lw.LW_FP64, det.n_pix, grid, want_X=True)
    got = lw.lw_spectrum_grad(traj, det, grid, X, torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    for name, g, o in zip(("r", "beta", "beta_dot"), got, ref):
        g = g.cpu().numpy()
        assert np.abs(o).max() > 0, name
        assert np.abs(g - o).max() <= 1e-9 * np.abs(o).max(), (name, np.abs(g - o).max(),
                                                               np.abs(o).max())


@pytest.mark.parametrize("precision", [lw.LW_MIXED_F32X4, lw.LW_MIXED])
@pytest.mark.parametrize("t_per_electron", [False, True])
def test_mixed_spectrum_grad_matches_oracle_gradient(t_per_electron, precision):
    """The mixed-precision adjoint (FP64 advanced times and bins, FP32 fields, weights and
    chain rule, X' from the mixed forward) against the oracle's chain-rule gradient:
    element-wise within 1e-4 of the largest element, 2e-5 relative L2 per array."""
    tr = simple.random_smooth(4, 90, 2e-18, 41, gamma=6.0, amp=0.4,
                              t_per_electron=t_per_electron)
    n_hat = _dirs(7, 5, 0.25)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    grid = lw.Grid(lo - 2.5 * (hi - lo) / 500, (hi - lo) / 500, 512)
    rng = np.random.Generator(np.random.PCG64(17))
    w = rng.uniform(0.2, 2.0, size=(7, 257))
    ref = oracle.tdm_grad(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, grid.t_min, grid.dt_u,
                          grid.n_bins, w)
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot,
                                     sections=lw.LW_SECTION_FP64 | lw.LW_SECTION_MIXED, block=32)
    det = lw.Detector(n_hat)
    rec = lw.lw_deposit_time_domain(traj, det, grid, precision)
    S, X = lw.lw_spectrum(rec, precision, det.n_pix, grid, want_X=True)
    assert X.dtype == torch.complex64
    got = lw.lw_spectrum_grad(traj, det, grid, X, torch.from_numpy(w).cuda(), precision=precision)
    torch.cuda.synchronize()
    for name, g, o in zip(("r", "beta", "beta_dot"), got, ref):
        g = g.cpu().numpy()
        assert np.all(np.isfinite(g)), name
        assert np.abs(g - o).max() <= 1e-4 * np.abs(o).max(), (name, np.abs(g - o).max(),
                                                               np.abs(o).max())
        assert np.linalg.norm(g - o) <= 2e-5 * np.linalg.norm(o), name


def _c4_small():
    laser = GaussianLaser(lam=1e-6, a0=1.0, w0=20e-6, fwhm=10e-15)
    n_e, gamma = 6, 60.0
    rng = np.random.Generator(np.random.PCG64(20603019))
    g = gamma * (1.0 + 1e-3 * rng.normal(size=n_e))
    uz = np.sqrt(g * g - 1.0)
    u0 = np.stack([np.zeros(n_e), np.zeros(n_e), uz], -1)
    sigma = laser.fwhm / (2.0 * math.sqrt(math.log(2.0)))
    t_half = 0.5 * sigma * math.sqrt(2.0 * math.log(1e6))
    # transverse offsets inside the waist so that w0 matters
    r0 = np.stack([rng.uniform(-8e-6, 8e-6, n_e), rng.uniform(-8e-6, 8e-6, n_e),
                   np.zeros(n_e)], -1) + (uz / g)[:, None] * np.array([0, 0, 299792458.0]) * -t_half
    return laser, r0, u0, -t_half, t_half, 800, gamma


def test_band_energy_gradient_wrt_initial_conditions_and_laser():
    laser, r0, u0, t0, t1, n_s, gamma = _c4_small()
    n_hat = _dirs(9, 11, 0.1 / gamma)
    tr0 = boris_trajectories(r0, u0, laser, t0, t1, n_s)
    lo, hi = oracle.grid_bounds(tr0.t, tr0.r, n_hat)
    # 4x zero padding; the grid starts half a bin before the earliest advanced time,
    # which otherwise lies exactly on grid point 0 (a kink of the loss at the
    # evaluation point itself, where only one-sided derivatives exist)
    dt_u = (hi - lo) / 2048
    grid = lw.Grid(lo - 0.5 * dt_u, dt_u, 8192)
    w1 = doppler_fundamental(gamma, laser.lam, laser.a0)
    mask = band_mask(grid, w1, 0.05).numpy()
    assert mask.sum() >= 8
    d_omega = 2 * math.pi / (grid.n_bins * grid.dt_u)
    det = lw.Detector(n_hat)
    dev = torch.device("cuda")
    u = torch.tensor(u0, device=dev, requires_grad=True)
    a0 = torch.tensor(laser.a0, dtype=torch.float64, device=dev, requires_grad=True)
    w0 = torch.tensor(laser.w0, dtype=torch.float64, device=dev, requires_grad=True)
    t, r, b, a = boris_push(torch.tensor(r0, device=dev), u, a0, w0, laser.lam, laser.fwhm, t0,
                            t1, n_s, checkpoint_every=256)
    S = LWSpectrum.apply(t, r, b, a, det, grid)
    L = band_energy(S, grid, torch.from_numpy(mask))
    L.backward()
    torch.cuda.synchronize()

    def L_oracle(u0_, a0_, w0_):
        """Loss and the grid interval index of every (direction, electron, sample)."""
        lz = GaussianLaser(lam=laser.lam, a0=a0_, w0=w0_, fwhm=laser.fwhm)
        tr = boris_trajectories(r0, u0_, lz, t0, t1, n_s)
        ta = oracle.advanced_times(tr.t, tr.r, n_hat)
        return (_oracle_loss(tr, n_hat, grid, mask[None, :] * d_omega),
                np.floor((ta - grid.t_min) / grid.dt_u))

    base, _ = L_oracle(u0, laser.a0, laser.w0)
    assert abs(float(L) / base - 1.0) < 1e-6     # torch and numpy pushers agree

    def kink_free_fd(shift, scale):
        for rel in (1e-7, 3e-8, 1e-8, 3e-9):
            h = rel * scale
            (Lp, jp), (Lm, jm) = L_oracle(*shift(h)), L_oracle(*shift(-h))
            if np.array_equal(jp, jm):
                return (Lp - Lm) / (2 * h)
        raise AssertionError("every stencil straddles a grid-point crossing")

    def shift_u(k, c):
        def f(h):
            v = u0.copy()
            v[k, c] += h
            return v, laser.a0, laser.w0
        return f

    # the same loss through the library's kernels only: GPU push, deposit, spectrum,
    # lw_spectrum_grad and the forward-mode push gradient
    u2 = torch.tensor(u0, device=dev, requires_grad=True)
    a2 = torch.tensor(laser.a0, dtype=torch.float64, device=dev, requires_grad=True)
    w2 = torch.tensor(laser.w0, dtype=torch.float64, device=dev, requires_grad=True)
    S2 = PushSpectrum.apply(u2, a2, w2, torch.tensor(r0, device=dev), laser.lam, laser.fwhm,
                            t0, t1, n_s, det, grid)
    L2 = band_energy(S2, grid, torch.from_numpy(mask))
    L2.backward()
    torch.cuda.synchronize()
    assert abs(float(L2) / float(L) - 1.0) < 1e-9
    assert float(torch.linalg.norm(u2.grad - u.grad) / torch.linalg.norm(u.grad)) < 1e-7
    checks = [(f"u0[{k},{c}]", (float(u.grad[k, c]), float(u2.grad[k, c])),
               kink_free_fd(shift_u(k, c), gamma)) for (k, c) in ((0, 2), (3, 0), (5, 2))]
    checks.append(("a0", (float(a0.grad), float(a2.grad)),
                   kink_free_fd(lambda h: (u0, laser.a0 + h, laser.w0), laser.a0)))
    checks.append(("w0", (float(w0.grad), float(w2.grad)),
                   kink_free_fd(lambda h: (u0, laser.a0, laser.w0 + h), laser.w0)))
    for name, gs, fd in checks:
        for g in gs:   # torch-autograd pusher, then the library's forward-mode kernel
            assert abs(g - fd) <= TOL * abs(fd), (name, g, fd)


def test_mixed_push_spectrum_gradient_matches_fp64():
    """Config 4's chain in mixed precision (mixed deposit and spectrum, mixed adjoint) against
    the FP64 chain on the small config-4 case: the loss within 1e-5, the gradients with
    respect to u0 (relative L2), a0 and w0 within 1e-4 (the FP64 chain is checked against
    finite differences of the oracle above)."""
    laser, r0, u0, t0, t1, n_s, gamma = _c4_small()
    n_hat = _dirs(9, 11, 0.1 / gamma)
    tr0 = boris_trajectories(r0, u0, laser, t0, t1, n_s)
    lo, hi = oracle.grid_bounds(tr0.t, tr0.r, n_hat)
    dt_u = (hi - lo) / 2048
    grid = lw.Grid(lo - 0.5 * dt_u, dt_u, 8192)
    mask = band_mask(grid, doppler_fundamental(gamma, laser.lam, laser.a0), 0.05)
    det = lw.Detector(n_hat)
    dev = torch.device("cuda")
    out = {}
    for prec in (lw.LW_FP64, lw.LW_MIXED_F32X4):
        u = torch.tensor(u0, device=dev, requires_grad=True)
        a0 = torch.tensor(laser.a0, dtype=torch.float64, device=dev, requires_grad=True)
        w0 = torch.tensor(laser.w0, dtype=torch.float64, device=dev, requires_grad=True)
        S = PushSpectrum.apply(u, a0, w0, torch.tensor(r0, device=dev), laser.lam, laser.fwhm,
                               t0, t1, n_s, det, grid, 1.602176634e-19, prec)
        L = band_energy(S.to(torch.float64), grid, mask)
        L.backward()
        torch.cuda.synchronize()
        out[prec] = (float(L), u.grad.clone(), float(a0.grad), float(w0.grad))
    L64, gu64, ga64, gw64 = out[lw.LW_FP64]
    L32, gu32, ga32, gw32 = out[lw.LW_MIXED_F32X4]
    assert abs(L32 / L64 - 1.0) < 1e-5
    assert float(torch.linalg.norm(gu32 - gu64) / torch.linalg.norm(gu64)) < 1e-4
    assert abs(ga32 - ga64) <= 1e-4 * abs(ga64)
    assert abs(gw32 - gw64) <= 1e-4 * abs(gw64)
