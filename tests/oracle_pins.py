"""Pins of the FP64 CPU oracle against facts that do not come from the oracle
itself: numbers printed in the paper, closed forms of classical
electrodynamics, invariants of the method and brute-force evaluation on tiny
inputs.  Each ``pin_*`` function raises AssertionError on failure and is
called by ``test_oracle_pins.py`` and, against deliberately broken builds of
the oracle, by ``test_oracle_mutations.py``.
"""
from __future__ import annotations

import math
import os

import numpy as np

import oracle
from oracle import estimates
from workloads import C0, EPS0, Q_E, detector_grid
from workloads import simple
from workloads.planewave import doppler_fundamental, plane_wave_trajectories

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def _rand_dirs(n, seed, max_angle=0.3):
    rng = np.random.Generator(np.random.PCG64(seed))
    tx = rng.uniform(-max_angle, max_angle, n)
    ty = rng.uniform(-max_angle, max_angle, n)
    return np.stack([np.sin(tx), np.cos(tx) * np.sin(ty), np.cos(tx) * np.cos(ty)], -1)


def _far_field_identity(n, beta, bdot):
    """n x ((n - beta) x bdot) / D^3 written through the BAC-CAB identity with |n| = 1:
    [(n - beta)(n . bdot) - D bdot] / D^3, D = 1 - n . beta (independent of the
    oracle's cross products)."""
    D = 1.0 - np.sum(n * beta, -1, keepdims=True)
    nb = np.sum(n * bdot, -1, keepdims=True)
    return ((n - beta) * nb - D * bdot) / D**3


# --------------------------------------------------------------- paper tables

def pin_table1_tu_estimation():
    """Table 1 (theory columns) of Sec. 4 with c0 = 0.3 um/fs."""
    for lx, ly, lz, T, g, tb, trad, tu in _rows("table1_tu_estimation.txt"):
        lx, ly, lz, T, g = map(float, (lx, ly, lz, T, g))
        assert abs(estimates.t_bunch_rad(lx, ly, lz, g, 0.3) - float(tb)) < 6e-5
        assert abs(estimates.t_rad(T, g) - float(trad)) < 1e-12
        assert abs(estimates.t_u_estimate(lx, ly, lz, T, g, 0.3) - float(tu)) < 6e-5


def pin_table2_ntu_ratio():
    """Table 2 of Sec. 4.2: 4 N_p / N_Tu to <= 0.1 % (printed to 4 digits)."""
    for name, E, lz, Q, T, lam, printed in _rows("table2_ntu_ratio.txt"):
        g = float(E) / 0.511
        n_p = float(Q) * 1e-12 / 1.6e-19
        ntu = estimates.n_tu_estimate(0.0, 0.0, float(lz) * 1e-6, float(T) * 1e-12, g,
                                      float(lam) * 1e-6, 3e8)
        ntu2 = estimates.n_tu_estimate_closed(0.0, 0.0, float(lz) * 1e-6, float(T) * 1e-12, g,
                                              float(lam) * 1e-6, 3e8)
        assert abs(ntu / ntu2 - 1.0) < 1e-12, name
        assert abs(4.0 * n_p / ntu / float(printed) - 1.0) < 1e-3, name


def pin_breakeven_exponent():
    """Sec. 5.2 worked example: exponent 2.5479e11 with the natural log."""
    g = {r[0]: float(r[1]) for r in _rows("performance_model.txt")}
    e = estimates.fdm_breakeven_exponent(g["C_omega"], g["C2_t"], g["N_s"], g["N_p"])
    assert abs(e / g["exponent"] - 1.0) < 5e-5


def pin_memory_model():
    """Eq. (parallel_scheme_function): both printed forms agree and phi >= 1
    exactly when N_obs N_Tu >= 4 N_p (Eq. parallel_scheme_function_2)."""
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(200):
        P = int(rng.integers(2, 512))
        n_p = float(rng.integers(1, 10**7))
        n_obs = float(rng.integers(1, 5000))
        n_tu = float(rng.integers(1, 10**6))
        a = estimates.phi_memory_ratio(P, n_p, n_obs, n_tu)
        b = estimates.phi_memory_ratio_expanded(P, n_p, n_obs, n_tu)
        assert abs(a / b - 1.0) < 1e-12
        assert (a >= 1.0) == (n_obs * n_tu - 4.0 * n_p >= 0.0) or abs(a - 1.0) < 1e-12


# --------------------------------------------------------------- deposit

def _membership(ta0, taN, t_min, dt_u, n_bins):
    j = np.arange(n_bins)
    tj = t_min + j * dt_u
    return (tj > ta0) & (tj <= taN)


def pin_stationary_constant_acceleration():
    """beta = 0, r = 0, constant beta_dot: t_a = t and F = (n.bdot) n - bdot is
    constant, so the record is exactly n_e F on the grid points in (t_0, t_N]."""
    tr = simple.stationary_constant_acceleration(57, 1.3e-18, (3e15, -2e15, 5e14), n_e=2,
                                                 t0=-2.0e-17)
    n_hat = _rand_dirs(5, 1)
    dt_u = 0.37 * 1.3e-18
    t_min = tr.t[0] - 5.21 * dt_u
    n_bins = 180
    rec, st = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, t_min, dt_u, n_bins)
    mask = _membership(tr.t[0], tr.t[-1], t_min, dt_u, n_bins)
    assert 100 < mask.sum() < n_bins
    for m in range(n_hat.shape[0]):
        F = _far_field_identity(n_hat[m], np.zeros(3), tr.beta_dot[0, 0])
        want = np.where(mask[None, :], 2.0 * F[:, None], 0.0)
        assert np.max(np.abs(rec[m] - want)) <= 1e-14 * np.abs(F).max()
    assert st == 0


def pin_linear_ramp():
    """beta_dot linear in t (beta = 0, r = 0): linear interpolation is exact,
    so rec(t_j) = F(t_j) at every covered grid point."""
    a0 = np.array([1e15, 4e14, -3e14])
    a1 = np.array([2e32, -5e31, 7e31])
    tr = simple.linear_ramp_acceleration(40, 2.0e-18, a0, a1, t0=0.0)
    n_hat = _rand_dirs(4, 2)
    dt_u = 0.61e-18
    t_min = -1.3e-18
    n_bins = 150
    rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, t_min, dt_u, n_bins)
    tj = t_min + np.arange(n_bins) * dt_u
    mask = _membership(tr.t[0], tr.t[-1], t_min, dt_u, n_bins)
    for m in range(n_hat.shape[0]):
        bd = a0[None, :] + a1[None, :] * tj[:, None]
        F = _far_field_identity(n_hat[m][None, :], np.zeros((1, 3)), bd)
        want = np.where(mask[:, None], F, 0.0).T
        scale = np.abs(F[mask]).max()
        assert np.max(np.abs(rec[m] - want)) <= 1e-13 * scale


def _moving_constant_field(n_e, n_s, seed, t_per_electron=False):
    """Positions from a smooth random trajectory but beta = 0 and a constant
    beta_dot, so F is constant while t_a follows the motion."""
    tr = simple.random_smooth(n_e, n_s, 3e-18, seed, gamma=8.0, amp=0.3,
                              t_per_electron=t_per_electron)
    beta = np.zeros_like(tr.r)
    bd = np.broadcast_to(np.array([2e15, 0.0, 0.0]), tr.r.shape).copy()
    return simple.Trajectories(tr.t, tr.r, beta, bd)


def pin_coverage_count():
    """Each (electron, pixel) pair deposits into exactly the grid points in
    (t_a(t_0), t_a(t_N)] (clipped): with a constant field the record divided
    by F counts the electrons covering each grid point."""
    tr = _moving_constant_field(5, 64, 11, t_per_electron=True)
    n_hat = _rand_dirs(3, 3, 0.4)
    ta = np.stack([tr.t - (n @ tr.r.transpose(0, 2, 1)) / C0 for n in n_hat])  # [m][k][i]
    lo, hi = ta[:, :, 0].min(), ta[:, :, -1].max()
    n_bins = 97
    dt_u = (hi - lo) / (n_bins - 20)
    t_min = lo - 7.3 * dt_u
    rec, st = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, t_min, dt_u, n_bins)
    for m in range(n_hat.shape[0]):
        F = _far_field_identity(n_hat[m], np.zeros(3), tr.beta_dot[0, 0])
        cover = sum(_membership(ta[m, k, 0], ta[m, k, -1], t_min, dt_u, n_bins).astype(float)
                    for k in range(tr.n_e))
        c = int(np.argmax(np.abs(F)))
        assert np.allclose(rec[m, c] / F[c], cover, atol=1e-12), m
    assert st & oracle.ST_CLIP == 0


def pin_linearity():
    """rec(A u B) = rec(A) + rec(B): superposition over electrons, which is
    also what beam-parallel sharding relies on."""
    tr = simple.random_smooth(5, 80, 2e-18, 21, gamma=6.0, amp=0.5)
    n_hat = _rand_dirs(4, 4, 0.2)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    n_bins = 256
    dt_u = (hi - lo) / n_bins
    args = (n_hat, lo, dt_u, n_bins)
    ra, _ = oracle.tdm_deposit(tr.t, tr.r[:3], tr.beta[:3], tr.beta_dot[:3], *args)
    rb, _ = oracle.tdm_deposit(tr.t, tr.r[3:], tr.beta[3:], tr.beta_dot[3:], *args)
    rab, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, *args)
    assert np.max(np.abs(rab - ra - rb)) <= 1e-12 * np.max(np.abs(rab))
    # transversality: every deposit is a combination of fields normal to n
    for m in range(n_hat.shape[0]):
        ndot = np.einsum("c,cj->j", n_hat[m], rab[m])
        assert np.max(np.abs(ndot)) <= 1e-12 * np.max(np.abs(rab[m]))


def brute_force_record(tr, n_hat, t_min, dt_u, n_bins):
    """Gather form of Algorithm 2 in plain Python: for each grid point t_j and
    electron, scan the steps for the interval with t_a(i-1) < t_j <= t_a(i) and
    interpolate linearly there.  Advanced times from Eq. (far_adv) and fields
    from the BAC-CAB form, both written independently of the oracle."""
    n_pix = n_hat.shape[0]
    out = np.zeros((n_pix, 3, n_bins))
    for m in range(n_pix):
        n = n_hat[m]
        for k in range(tr.n_e):
            t = tr.t if tr.t.ndim == 1 else tr.t[k]
            ta = [float(t[i]) - float(n @ tr.r[k, i]) / C0 for i in range(tr.n_s + 1)]
            F = _far_field_identity(n[None, :], tr.beta[k], tr.beta_dot[k])
            for j in range(n_bins):
                tj = t_min + j * dt_u
                for i in range(1, tr.n_s + 1):
                    if ta[i - 1] < tj <= ta[i]:
                        w = (tj - ta[i - 1]) / (ta[i] - ta[i - 1])
                        out[m, :, j] += F[i - 1] * (1.0 - w) + F[i] * w
    return out


def pin_brute_force_tiny():
    """Oracle deposit == brute-force gather on tiny ragged inputs (shared and
    per-electron time axes)."""
    for per_e, seed in ((False, 31), (True, 32)):
        tr = simple.random_smooth(3, 23, 4e-18, seed, gamma=5.0, amp=0.6, t_per_electron=per_e)
        n_hat = _rand_dirs(3, seed, 0.3)
        lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
        n_bins = 37
        dt_u = (hi - lo) / 30.3
        t_min = lo - 2.7 * dt_u
        rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, t_min, dt_u, n_bins)
        ref = brute_force_record(tr, n_hat, t_min, dt_u, n_bins)
        assert np.max(np.abs(rec - ref)) <= 1e-11 * np.max(np.abs(ref)), per_e


def pin_grid_bounds():
    """Eqs. (tu_min), (tu_max) use only the first and last samples; for
    physical trajectories t_a is increasing, so they equal the brute min/max
    over all samples."""
    tr = simple.random_smooth(6, 50, 3e-18, 41, gamma=4.0, amp=0.5)
    n_hat = _rand_dirs(7, 5, 0.5)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    ta = np.stack([tr.t[None, :] - (tr.r @ n) / C0 for n in n_hat])
    assert np.all(np.diff(ta, axis=-1) > 0)
    assert abs(lo - ta.min()) <= 1e-30 + 1e-15 * abs(lo)
    assert abs(hi - ta.max()) <= 1e-30 + 1e-15 * abs(hi)
    ta_o = oracle.advanced_times(tr.t, tr.r, n_hat)
    assert np.allclose(ta_o, ta, rtol=0, atol=1e-15 * np.abs(ta).max())


def pin_far_vs_exact_time():
    """Far-field time map vs the exact advanced condition (Eq. advanced_condition):
    t_a_exact - R/c0 - t_a_far = O(|x'|^2 / (R c0))."""
    tr = simple.random_smooth(2, 20, 3e-18, 51, gamma=3.0, amp=0.4, spread=1e-6)
    n_hat = _rand_dirs(4, 6, 0.5)
    R = 0.5
    far = oracle.advanced_times(tr.t, tr.r, n_hat, R=R)
    ex = oracle.advanced_times(tr.t, tr.r, n_hat, R=R, flags=oracle.FLAG_EXACT)
    bound = np.max(np.sum(tr.r**2, -1)) / (R * C0)
    assert np.max(np.abs(ex - R / C0 - far)) <= bound + 1e-24


# --------------------------------------------------------------- FFT and spectrum

def pin_fft_vs_dft_and_convention():
    """FFT == direct DFT; a single complex exponential exp(-2 pi i j l0/N)
    maps to N at bin l0 (this fixes the exp(+j omega t) sign of Eq. efield_xfrom);
    discrete Parseval."""
    rng = np.random.Generator(np.random.PCG64(7))
    for n in (1, 2, 4, 8, 64, 256, 1024):
        x = rng.normal(size=n) + 1j * rng.normal(size=n)
        X = oracle.fft(x)
        Xd = oracle.dft(x)
        assert np.max(np.abs(X - Xd)) <= 1e-12 * max(1.0, np.abs(Xd).max())
        assert abs(np.sum(np.abs(X) ** 2) - n * np.sum(np.abs(x) ** 2)) <= 1e-10 * n * np.sum(
            np.abs(x) ** 2)
    for n, l0 in ((16, 3), (128, 45), (64, 0)):
        j = np.arange(n)
        for f in (oracle.fft, oracle.dft):
            X = f(np.exp(-2j * np.pi * j * l0 / n))
            want = np.zeros(n, complex)
            want[l0] = n
            assert np.max(np.abs(X - want)) <= 1e-9


def pin_spectrum_cosine_line():
    """A pure cosine record at bin l0 gives a single spectral line of height
    q^2 dt_u^2 (N/2)^2 / (16 pi^3 eps0 c0) per unit-amplitude component."""
    n, l0, dt_u = 256, 19, 3e-18
    j = np.arange(n)
    rec = np.zeros((1, 3, n))
    rec[0, 1] = np.cos(2 * np.pi * l0 * j / n)
    S = oracle.spectrum(rec, dt_u)
    K = Q_E**2 / (16.0 * math.pi**3 * EPS0 * C0)
    want = np.zeros(n // 2 + 1)
    want[l0] = K * dt_u**2 * (n / 2) ** 2
    assert np.max(np.abs(S[0] - want)) <= 1e-10 * want.max()


def pin_spectrum_parseval():
    """Physical Parseval: sum over the full spectrum of S_l d_omega equals
    2 pi K dt_u sum_j |rec_j|^2 (K = q^2/(16 pi^3 eps0 c0))."""
    rng = np.random.Generator(np.random.PCG64(8))
    n, dt_u = 512, 2.5e-18
    rec = rng.normal(size=(2, 3, n))
    S = oracle.spectrum(rec, dt_u)
    d_omega = 2 * math.pi / (n * dt_u)
    full = S[:, 0] + 2.0 * S[:, 1:-1].sum(-1) + S[:, -1]
    K = Q_E**2 / (16.0 * math.pi**3 * EPS0 * C0)
    want = 2 * math.pi * K * dt_u * np.sum(rec**2, axis=(1, 2))
    assert np.allclose(full * d_omega, want, rtol=1e-11)


# --------------------------------------------------------------- physics closed forms

def _coulomb_error(n_s):
    beta = 0.6
    R = 1e-6
    n_hat = np.array([[1.0, 0.0, 0.0]])
    T = 40e-15
    tr = simple.uniform_motion(n_s, 2 * T / n_s, (0.0, 0.0, beta), t0=-T)
    flags = oracle.FLAG_EXACT | oracle.FLAG_VELOCITY
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat, R=R, flags=flags)
    n_bins = 64
    t_min = lo + 0.25 * (hi - lo)
    dt_u = 0.5 * (hi - lo) / n_bins
    rec, st = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, t_min, dt_u, n_bins,
                                 R=R, flags=flags)
    assert st & ~oracle.ST_CLIP == 0
    tj = t_min + dt_u * np.arange(n_bins)
    obs = R * n_hat[0]
    present = np.stack([np.zeros_like(tj), np.zeros_like(tj), beta * C0 * tj], -1)
    Rp = obs[None, :] - present
    Rn = np.linalg.norm(Rp, axis=-1)
    sin2 = 1.0 - (Rp[:, 2] / Rn) ** 2
    g2inv = 1.0 - beta**2
    # q (1 - beta^2) / (4 pi eps0 Rp^2 (1 - beta^2 sin^2 psi)^{3/2}) R_hat, times 4 pi eps0 c0 R / q
    E = (C0 * R * g2inv / (Rn**2 * (1.0 - beta**2 * sin2) ** 1.5))[:, None] * (Rp / Rn[:, None])
    return np.max(np.abs(rec[0].T - E)) / np.max(np.abs(E))


def pin_boosted_coulomb():
    """Exact geometry with the velocity field, uniform motion: the record at
    observer time t_j equals the boosted Coulomb field of the charge's present
    position (Jackson Eq. 11.154 form), with second-order convergence in dt."""
    e1 = _coulomb_error(400)
    e2 = _coulomb_error(1600)
    assert e1 < 2e-3 and e2 < 1e-4
    assert 10.0 < e1 / e2 < 25.0, (e1, e2)     # 4x finer steps -> ~16x smaller error


def pin_larmor_total_energy():
    """Energy received over the full sphere equals the Lienard-Larmor energy
    emitted, int P dt with P = q^2 gamma^6 (|bdot|^2 - |beta x bdot|^2)/(6 pi eps0 c0),
    computed from the spectra S (one-sided integral over omega) with the
    paper's solid-angle parametrisation d_Omega = cos(theta_x) d_theta_x d_theta_y."""
    beta0, omega = 0.5, 2.0e15
    n_s = 1200
    T = 4 * 2 * math.pi / omega
    tr = simple.circular_motion(n_s, T / n_s, beta0, omega)
    ntx, nty = 24, 48
    tx = (np.arange(ntx) + 0.5) / ntx * math.pi - math.pi / 2
    ty = (np.arange(nty) + 0.5) / nty * 2 * math.pi - math.pi
    TX, TY = np.meshgrid(tx, ty, indexing="ij")
    TX, TY = TX.ravel(), TY.ravel()
    n_hat = np.stack([np.sin(TX), np.cos(TX) * np.sin(TY), np.cos(TX) * np.cos(TY)], -1)
    dOmega = np.cos(TX) * (math.pi / ntx) * (2 * math.pi / nty)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    n_bins = 4096
    dt_u = (hi - lo) / (n_bins - 4)
    t_min = lo - 2 * dt_u
    rec, st = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, t_min, dt_u, n_bins)
    S = oracle.spectrum(rec, dt_u)
    d_omega = 2 * math.pi / (n_bins * dt_u)
    dW = (0.5 * S[:, 0] + S[:, 1:-1].sum(-1) + 0.5 * S[:, -1]) * d_omega
    total = float(np.sum(dW * dOmega))
    g = 1.0 / math.sqrt(1 - beta0**2)
    P = Q_E**2 * g**6 * (beta0**2 * omega**2 - beta0**4 * omega**2) / (6 * math.pi * EPS0 * C0)
    assert abs(total / (P * T) - 1.0) < 5e-3, total / (P * T)


def _on_axis_spectrum(gamma, a0, fwhm, n_s, n_bins, lam=1e-6, pad=1):
    sigma = fwhm / (2 * math.sqrt(math.log(2)))
    th = 0.5 * sigma * math.sqrt(2 * math.log(1e6))
    tr = plane_wave_trajectories(gamma, lam, a0, fwhm, -th, th, n_s)
    n_hat = np.array([[0.0, 0.0, 1.0]])
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    dt_u = (hi - lo) / n_bins
    n_tot = n_bins * pad                       # zero padding refines the frequency grid
    rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, lo, dt_u, n_tot)
    S = oracle.spectrum(rec, dt_u)[0]
    w = 2 * math.pi * np.arange(n_tot // 2 + 1) / (n_tot * dt_u)
    return w, S


def pin_doppler_line():
    """On-axis inverse Compton line omega_1 = 4 gamma^2 omega_L / (1 + a0^2/2):
    for a0 = 0.1 (long pulse) the line centroid is within 1 % of omega_1; for
    a0 = 0.5 the line is chirped by the envelope, its red half-maximum edge
    sits within 1.5 % of omega_1(a0) (an 11 % red shift) and its blue edge
    (last point above 1 % of the peak) within 2 % of omega_1(a0 = 0)."""
    g = 10.0
    w, S = _on_axis_spectrum(g, 0.1, 100e-15, 4000, 4096)
    w1 = doppler_fundamental(g, 1e-6, 0.1)
    band = (w > 0.5 * w1) & (w < 1.5 * w1)
    cen = np.sum(w[band] * S[band]) / np.sum(S[band])
    assert abs(cen / w1 - 1.0) < 1e-2, cen / w1
    w, S = _on_axis_spectrum(g, 0.5, 100e-15, 4000, 4096, pad=8)
    w1 = doppler_fundamental(g, 1e-6, 0.5)
    w0 = doppler_fundamental(g, 1e-6, 0.0)
    band = (w > 0.5 * w1) & (w < 1.5 * w1)
    wb, Sb = w[band], S[band] / S[band].max()
    ipk = int(np.argmax(Sb))
    red = wb[:ipk][Sb[:ipk] < 0.5][-1]
    blue = wb[Sb > 1e-2][-1]
    assert abs(red / w1 - 1.0) < 1.5e-2, red / w1
    assert abs(blue / w0 - 1.0) < 2e-2, blue / w0


def pin_coherence():
    """N identical electrons radiate N^2 times the single-electron spectrum."""
    tr = plane_wave_trajectories(8.0, 1e-6, 0.2, 20e-15, -40e-15, 40e-15, 600, n_e=1)
    tr4 = simple.Trajectories(tr.t, np.repeat(tr.r, 4, 0), np.repeat(tr.beta, 4, 0),
                              np.repeat(tr.beta_dot, 4, 0))
    n_hat = _rand_dirs(3, 9, 0.05)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    dt_u = (hi - lo) / 1024
    r1, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, lo, dt_u, 1024)
    r4, _ = oracle.tdm_deposit(tr4.t, tr4.r, tr4.beta, tr4.beta_dot, n_hat, lo, dt_u, 1024)
    assert np.max(np.abs(r4 - 4 * r1)) <= 1e-14 * np.max(np.abs(r4))
    S1 = oracle.spectrum(r1, dt_u)
    S4 = oracle.spectrum(r4, dt_u)
    assert np.max(np.abs(S4 - 16 * S1)) <= 1e-12 * np.max(S4)


def pin_fdm_vs_tdm():
    """The paper's two methods agree on a Nyquist-resolved case (gamma = 5,
    plane wave): the normalised error of Eq. (spectra_error) between TDM and
    the FDM of Eq. (inty_dft) at the TDM frequencies has a mean below 1e-2 and
    a maximum below 0.13 (the levels of the paper's accuracy tables)."""
    g = 5.0
    tr = plane_wave_trajectories(g, 1e-6, 0.2, 25e-15, -60e-15, 60e-15, 3000)
    n_hat = _rand_dirs(3, 10, 0.4 / g)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    n_bins = 2048
    dt_u = (hi - lo) / n_bins
    rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, lo, dt_u, n_bins)
    S_t = oracle.spectrum(rec, dt_u)
    w = 2 * math.pi * np.arange(n_bins // 2 + 1) / (n_bins * dt_u)
    w1 = doppler_fundamental(g, 1e-6, 0.2)
    sel = np.nonzero(w < 3.0 * w1)[0]
    S_f, _ = oracle.fdm(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, w[sel], tr.t[1] - tr.t[0])
    err = np.abs(S_t[:, sel] - S_f) / S_f.max()
    assert err.mean() < 1e-2 and err.max() < 0.13, (err.mean(), err.max())


def pin_status_bits():
    """Clipping, non-increasing lab time, |beta| >= 1 and non-finite inputs are
    reported through the status word."""
    tr = simple.stationary_constant_acceleration(20, 1e-18, (1e15, 0, 0))
    n_hat = _rand_dirs(2, 12)
    # grid starting inside the trajectory's arrival window: low-side clipping only
    _, st = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, tr.t[0] + 5.5e-18,
                               1e-18, 64)
    assert st == oracle.ST_CLIP
    # grid ending inside the window: high-side clipping only
    _, st = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, tr.t[0] - 0.5e-18,
                               1e-18, 6)
    assert st == oracle.ST_CLIP
    _, st = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, tr.t[0] - 0.5e-18,
                               1e-18, 64)
    assert st == 0
    t = tr.t.copy()
    t[7] = t[6]
    _, st = oracle.tdm_deposit(t, tr.r, tr.beta, tr.beta_dot, n_hat, tr.t[0], 1e-18, 64)
    assert st & oracle.ST_TIME
    b = tr.beta.copy()
    b[0, 3] = (0.0, 0.0, 1.0)
    _, st = oracle.tdm_deposit(tr.t, tr.r, b, tr.beta_dot, n_hat, tr.t[0], 1e-18, 64)
    assert st & oracle.ST_BETA
    r = tr.r.copy()
    r[0, 5, 1] = np.nan
    _, st = oracle.tdm_deposit(tr.t, r, tr.beta, tr.beta_dot, n_hat, tr.t[0], 1e-18, 64)
    assert st & oracle.ST_NONFINITE


def pin_gradient_central_differences():
    """The oracle's gradient of L = sum g S (oracle.tdm_grad) against central differences
    of the oracle's own loss, per input element: position, velocity, acceleration of
    samples (the four largest gradients of each array and one of median size), to 1e-3 of
    the difference quotient (steps of 1e-6 of each array's scale; the loss is piecewise
    smooth, so a stencil near a grid-point crossing measures the slope to about that)."""
    tr = simple.random_smooth(3, 60, 2e-18, 301, gamma=5.0, amp=0.5)
    n_hat = _rand_dirs(5, 7, 0.3)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    n_bins = 256
    dt_u = (hi - lo) / 250
    t_min = lo - 3 * dt_u
    rng = np.random.Generator(np.random.PCG64(9))
    g = rng.uniform(0.5, 1.5, size=(5, n_bins // 2 + 1))
    grads = oracle.tdm_grad(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, t_min, dt_u, n_bins, g)

    def loss(r, b, a):
        rec, _ = oracle.tdm_deposit(tr.t, r, b, a, n_hat, t_min, dt_u, n_bins)
        return float(np.sum(g * oracle.spectrum(rec, dt_u)))

    base = [tr.r, tr.beta, tr.beta_dot]
    for which in range(3):
        h = 1e-6 * np.abs(base[which]).max()
        ga = np.abs(grads[which])
        gmax = ga.max()
        assert gmax > 0
        # the four largest elements and one of median size among the nonzero ones
        flat = np.argsort(ga.ravel())
        nz = flat[ga.ravel()[flat] > 0]
        picks = list(flat[-4:]) + [nz[len(nz) // 2]]
        for (k, i, c) in (np.unravel_index(f, ga.shape) for f in picks):
            plus = [x.copy() for x in base]
            minus = [x.copy() for x in base]
            plus[which][k, i, c] += h
            minus[which][k, i, c] -= h
            fd = (loss(*plus) - loss(*minus)) / (2 * h)
            assert abs(grads[which][k, i, c] - fd) <= 1e-3 * max(abs(fd), 1e-3 * gmax), \
                (which, k, i, c, grads[which][k, i, c], fd)


ALL_PINS = [
    pin_table1_tu_estimation,
    pin_table2_ntu_ratio,
    pin_breakeven_exponent,
    pin_memory_model,
    pin_stationary_constant_acceleration,
    pin_linear_ramp,
    pin_coverage_count,
    pin_linearity,
    pin_brute_force_tiny,
    pin_grid_bounds,
    pin_far_vs_exact_time,
    pin_fft_vs_dft_and_convention,
    pin_spectrum_cosine_line,
    pin_spectrum_parseval,
    pin_boosted_coulomb,
    pin_larmor_total_energy,
    pin_doppler_line,
    pin_coherence,
    pin_fdm_vs_tdm,
    pin_status_bits,
    pin_gradient_central_differences,
]
