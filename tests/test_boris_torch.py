"""The differentiable torch Boris pusher reproduces the workload generator's
numpy pusher (same algorithm), and its checkpointed autograd gradient matches
finite differences of a smooth functional (CPU)."""
import numpy as np
import torch

from paper_2206_03015_gb300.autograd import boris_push
from workloads.boris import GaussianLaser, boris_trajectories


def _setup(n_e=3, n_s=300):
    laser = GaussianLaser(lam=1e-6, a0=0.8, w0=15e-6, fwhm=10e-15)
    rng = np.random.Generator(np.random.PCG64(1))
    r0 = rng.normal(size=(n_e, 3)) * 1e-6 + np.array([0, 0, -4.7e-6])
    u0 = np.stack([rng.normal(size=n_e) * 0.05, rng.normal(size=n_e) * 0.05,
                   40.0 + rng.normal(size=n_e)], -1)
    return laser, r0, u0, -16e-15, 16e-15, n_s


def test_torch_pusher_matches_numpy_generator():
    laser, r0, u0, t0, t1, n_s = _setup()
    ref = boris_trajectories(r0, u0, laser, t0, t1, n_s)
    f64 = torch.float64
    t, r, b, a = boris_push(torch.tensor(r0), torch.tensor(u0), torch.tensor(laser.a0, dtype=f64),
                            torch.tensor(laser.w0, dtype=f64), laser.lam, laser.fwhm, t0, t1,
                            n_s, checkpoint_every=64)
    # same algorithm; only the rounding order of library routines differs
    assert np.allclose(t.numpy(), ref.t, rtol=0, atol=1e-27)
    assert np.max(np.abs(r.numpy() - ref.r)) <= 1e-10 * np.max(np.abs(ref.r))
    assert np.max(np.abs(b.numpy() - ref.beta)) <= 1e-10
    assert np.max(np.abs(a.numpy() - ref.beta_dot)) <= 1e-8 * np.max(np.abs(ref.beta_dot))


def test_checkpointed_gradient_matches_finite_differences():
    laser, r0, u0, t0, t1, n_s = _setup(n_e=2, n_s=200)

    def functional(u0_t, a0_t, w0_t):
        _, r, b, a = boris_push(torch.tensor(r0), u0_t, a0_t, w0_t, laser.lam, laser.fwhm, t0,
                                t1, n_s, checkpoint_every=50)
        return (a[..., 0] ** 2).sum() * 1e-30 + (r[..., 0] ** 2).sum() * 1e12

    u = torch.tensor(u0, requires_grad=True)
    a0 = torch.tensor(laser.a0, dtype=torch.float64, requires_grad=True)
    w0 = torch.tensor(laser.w0, dtype=torch.float64, requires_grad=True)
    L = functional(u, a0, w0)
    L.backward()
    for (name, x, idx, h) in (("u0x", u, (0, 0), 1e-6), ("u0z", u, (1, 2), 1e-5),
                              ("a0", a0, (), 1e-7), ("w0", w0, (), 1e-9)):
        with torch.no_grad():
            xp = x.detach().clone()
            xm = x.detach().clone()
            xp[idx] += h
            xm[idx] -= h
            args_p = [u.detach(), a0.detach(), w0.detach()]
            args_m = [u.detach(), a0.detach(), w0.detach()]
            k = {"u0x": 0, "u0z": 0, "a0": 1, "w0": 2}[name]
            args_p[k] = xp
            args_m[k] = xm
            fd = (functional(*args_p) - functional(*args_m)) / (2 * h)
        g = x.grad[idx]
        assert abs(float(g) - float(fd)) <= 1e-4 * max(abs(float(fd)), 1e-30), (name, g, fd)
