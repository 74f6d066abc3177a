"""CUDA path (through the C ABI) against the CPU oracle, element by element,
on seeded inputs that span several tiles and ragged tails, plus edge cases.

Tolerances: FP64 path 1e-9 relative L2 (records and spectra); the advanced
times and bin indices are bit-identical by construction, so the observed
error is summation order only (~1e-15).  Mixed path 1e-4 relative L2 on
spectra (FP32 field and FFT, FP64-exact bin coordinates)."""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_cases import gpu_bounds, gpu_run, oracle_run, rel_l2
from paper_2206_03015_gb300 import lw
from workloads import configs, simple

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
MIXED_TOL = 1e-4


def _dirs(n, seed, max_angle):
    rng = np.random.Generator(np.random.PCG64(seed))
    tx = rng.uniform(-max_angle, max_angle, n)
    ty = rng.uniform(-max_angle, max_angle, n)
    return np.stack([np.sin(tx), np.cos(tx) * np.sin(ty), np.cos(tx) * np.cos(ty)], -1)


def _case(name):
    """(trajectories, n_hat, grid, flags, R) for the named parity case."""
    if name == "ragged":           # 3 electrons x 38 samples, 129 pixels, 300 bins, clipping
        tr = simple.random_smooth(3, 37, 3e-18, 101, gamma=6.0, amp=0.5)
        n_hat = _dirs(129, 1, 0.2)
        lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
        grid = lw.Grid(lo + 0.1 * (hi - lo), (hi - lo) / 280.0, 300)
        return tr, n_hat, grid, lw.LW_FIELD_ACCEL, 1.0
    if name == "t_per_electron":
        tr = simple.random_smooth(5, 150, 2e-18, 102, gamma=4.0, amp=0.4, t_per_electron=True)
        n_hat = _dirs(77, 2, 0.3)
        lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
        grid = lw.Grid(lo, (hi - lo) / 512, 512)
        return tr, n_hat, grid, lw.LW_FIELD_ACCEL, 1.0
    if name == "velocity_field":
        tr = simple.random_smooth(4, 200, 2e-18, 103, gamma=3.0, amp=0.5)
        n_hat = _dirs(64, 3, 0.5)
        lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
        grid = lw.Grid(lo, (hi - lo) / 1024, 1024)
        return tr, n_hat, grid, lw.LW_FIELD_ACCEL | lw.LW_FIELD_VELOCITY, 1e-4
    if name == "many_bins_per_step":   # b >> 1: each step covers many grid points
        tr = simple.random_smooth(2, 40, 5e-18, 104, gamma=2.0, amp=0.5)
        n_hat = _dirs(33, 4, 0.4)
        lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
        grid = lw.Grid(lo, (hi - lo) / 4096, 4096)
        return tr, n_hat, grid, lw.LW_FIELD_ACCEL, 1.0
    if name == "c1_small":             # C1 physics at reduced size
        w = configs.c1_tiny(n_e=16, n_s=2000, nx=8, n_bins=4096)
        lo, hi = oracle.grid_bounds(w.traj.t, w.traj.r, w.n_hat)
        return w.traj, w.n_hat, lw.grid_from_bounds(lo, hi, 4096), lw.LW_FIELD_ACCEL, 1.0
    if name == "c1_offsets":
        w = configs.c1_offsets(n_e=16, n_s=2000, nx=8, n_bins=4096)
        lo, hi = oracle.grid_bounds(w.traj.t, w.traj.r, w.n_hat)
        return w.traj, w.n_hat, lw.grid_from_bounds(lo, hi, 4096), lw.LW_FIELD_ACCEL, 1.0
    if name == "single":               # degenerate: one electron, one step, one pixel, one bin
        tr = simple.stationary_constant_acceleration(1, 1e-18, (1e15, 2e15, 0.0), t0=0.0)
        n_hat = np.array([[0.0, 0.0, 1.0]])
        return tr, n_hat, lw.Grid(0.5e-18, 1e-18, 1), lw.LW_FIELD_ACCEL, 1.0
    if name == "all_clipped":          # grid after the whole arrival window
        tr = simple.random_smooth(2, 30, 3e-18, 105, gamma=5.0)
        n_hat = _dirs(5, 5, 0.2)
        lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
        return tr, n_hat, lw.Grid(hi + (hi - lo), (hi - lo) / 64, 64), lw.LW_FIELD_ACCEL, 1.0
    raise KeyError(name)


CASES = ["ragged", "t_per_electron", "velocity_field", "many_bins_per_step", "c1_small",
         "c1_offsets", "single", "all_clipped"]


@pytest.mark.parametrize("name", CASES)
def test_grid_bounds_bit_exact(name):
    tr, n_hat, _, _, _ = _case(name)
    assert gpu_bounds(tr, n_hat) == oracle.grid_bounds(tr.t, tr.r, n_hat)


@pytest.mark.parametrize("name", CASES)
def test_fp64_record_and_spectrum(name):
    tr, n_hat, grid, flags, R = _case(name)
    g = gpu_run(tr, n_hat, grid, lw.LW_FP64, flags, R)
    o = oracle_run(tr, n_hat, grid, flags, R)
    assert g["status"] == o["status"]
    scale = max(np.abs(o["rec"]).max(), 1e-300)
    assert np.max(np.abs(g["rec"] - o["rec"])) <= 1e-12 * scale
    assert rel_l2(g["rec"], o["rec"]) <= FP64_TOL
    if "S" in o:
        assert rel_l2(g["S"], o["S"]) <= FP64_TOL


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("block", [16, 128, 1024])
@pytest.mark.parametrize("precision", [lw.LW_MIXED, lw.LW_MIXED_KAHAN, lw.LW_MIXED_F32,
                                       lw.LW_MIXED_F32X4])
def test_mixed_record_and_spectrum(name, block, precision):
    tr, n_hat, grid, flags, R = _case(name)
    g = gpu_run(tr, n_hat, grid, precision, flags, R, block=block)
    o = oracle_run(tr, n_hat, grid, flags, R)
    # the mixed path reports input faults like the oracle; CLIP can differ when the last
    # arrival lies within FP32 rounding of a grid point, and it does not report TA_ORDER
    ignore = oracle.ST_TA_ORDER | oracle.ST_CLIP
    assert (g["status"] & ~ignore) == (o["status"] & ~ignore)
    if np.abs(o["rec"]).max() == 0:
        assert np.abs(g["rec"]).max() == 0
        return
    assert rel_l2(g["rec"], o["rec"]) <= MIXED_TOL
    if "S" in o:
        assert rel_l2(g["S"], o["S"]) <= MIXED_TOL


@pytest.mark.parametrize("n_bins", [2, 4, 64, 1024, 4096, 8192, 65536, 131072])
@pytest.mark.parametrize("n_pix", [1, 2, 5])
def test_spectrum_matches_oracle(n_bins, n_pix):
    rng = np.random.Generator(np.random.PCG64(n_bins + n_pix))
    rec = rng.normal(size=(n_pix, 3, n_bins)) * 1e20
    dt_u = 3.7e-18
    grid = lw.Grid(0.0, dt_u, n_bins)
    S_o, X_o = oracle.spectrum(rec, dt_u, want_X=True)
    K = 1.602176634e-19**2 / (16 * math.pi**3 * 8.8541878128e-12 * 299792458.0)
    X_o = X_o * math.sqrt(K) * dt_u
    S_g, X_g = lw.lw_spectrum(torch.from_numpy(rec).cuda(), lw.LW_FP64, n_pix, grid, want_X=True)
    assert rel_l2(S_g.cpu().numpy(), S_o) <= 1e-12
    assert rel_l2(X_g.cpu().numpy(), X_o) <= 1e-12
    rec32 = np.stack([rec.astype(np.float32), np.zeros_like(rec, dtype=np.float32)], -1)
    S_k = lw.lw_spectrum(torch.from_numpy(rec32).cuda(), lw.LW_MIXED_KAHAN, n_pix, grid)
    assert rel_l2(S_k.double().cpu().numpy(), S_o) <= 1e-5
    S_m = lw.lw_spectrum(torch.from_numpy(rec).cuda(), lw.LW_MIXED, n_pix, grid)
    assert rel_l2(S_m.double().cpu().numpy(), S_o) <= 1e-5
    S_f = lw.lw_spectrum(torch.from_numpy(rec.astype(np.float32)).cuda(), lw.LW_MIXED_F32,
                         n_pix, grid)
    assert rel_l2(S_f.double().cpu().numpy(), S_o) <= 1e-5
    rec4 = np.zeros((n_pix, n_bins, 4), dtype=np.float32)
    rec4[..., :3] = rec.transpose(0, 2, 1)
    rec4[..., 3] = 1e30   # the fourth lane is never read
    S_4 = lw.lw_spectrum(torch.from_numpy(rec4).cuda(), lw.LW_MIXED_F32X4, n_pix, grid)
    assert rel_l2(S_4.double().cpu().numpy(), S_o) <= 1e-5


def test_status_word_reports_bad_inputs():
    tr = simple.stationary_constant_acceleration(20, 1e-18, (1e15, 0.0, 0.0))
    n_hat = np.array([[0.0, 0.1, math.sqrt(1 - 0.01)]])
    b = tr.beta.copy()
    b[0, 3] = (0.0, 0.0, 1.0)
    t = tr.t.copy()
    t[7] = t[6]
    bad = simple.Trajectories(t, tr.r, b, tr.beta_dot)
    grid = lw.Grid(tr.t[0], 1e-18, 64)
    for prec in (lw.LW_FP64, lw.LW_MIXED, lw.LW_MIXED_KAHAN, lw.LW_MIXED_F32,
                 lw.LW_MIXED_F32X4):
        g = gpu_run(bad, n_hat, grid, prec, spectrum=False)
        assert g["status"] & lw.LW_ST_BETA and g["status"] & lw.LW_ST_TIME


def test_upload_orders_electrons_by_first_light_front_time():
    """The mixed section's electron order is a permutation sorted by buckets of
    1/4096 of the range of tau = t - z/c0 at the first sample."""
    tr = simple.random_smooth(300, 40, 2e-18, 61, gamma=8.0, amp=0.3)
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot)
    order = traj.order().cpu().numpy()
    assert np.array_equal(np.sort(order), np.arange(tr.n_e))
    t0 = tr.t[0] if tr.t.ndim == 1 else tr.t[:, 0]
    tau = t0 - tr.r[:, 0, 2] * (1.0 / 299792458.0)
    lo, hi = tau.min(), tau.max()
    bucket = np.minimum(((tau - lo) / (hi - lo) * 4096).astype(np.int64), 4095)
    # the device may round tau differently by an ulp (FMA), moving a key across a
    # bucket edge: allow one bucket of disorder, nothing more
    assert np.all(np.diff(bucket[order]) >= -1)
    assert np.mean(np.diff(bucket[order]) >= 0) > 0.99
    # uploads with the FP64 section only are ordered too (the order inside a bucket
    # follows the atomics, so only the buckets' sequence is fixed)
    other = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot,
                                      sections=lw.LW_SECTION_FP64).order().cpu().numpy()
    assert np.array_equal(np.sort(other), np.arange(tr.n_e))
    assert np.all(np.diff(bucket[other]) >= -1)


@pytest.mark.parametrize("precision", [lw.LW_FP64, lw.LW_MIXED])
def test_electron_chunks_accumulate_to_the_whole_deposit(precision):
    """The record is a sum over electrons: depositing electron chunks from pinned host
    inputs into one record (accumulate) equals one deposit of all electrons from
    device inputs, up to the order of the FP64 additions."""
    tr, n_hat, grid, flags, R = _case("c1_offsets")
    det = lw.Detector(n_hat)
    whole = lw.lw_deposit_time_domain(lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot),
                                      det, grid, precision)
    h = [torch.from_numpy(x).pin_memory() for x in (tr.t, tr.r, tr.beta, tr.beta_dot)]
    shp, dt = lw.record_shape(det, grid, precision)
    rec = torch.zeros(shp, dtype=dt, device="cuda")
    cuts = [0, 3, 4, 11, tr.n_e]
    for k0, k1 in zip(cuts[:-1], cuts[1:]):
        part = lw.lw_trajectories_upload(h[0], h[1][k0:k1], h[2][k0:k1], h[3][k0:k1])
        lw.lw_deposit_time_domain(part, det, grid, precision, record=rec, accumulate=True)
    torch.cuda.synchronize()
    a = lw.record_value(rec, precision).cpu().numpy()
    b = lw.record_value(whole, precision).cpu().numpy()
    assert rel_l2(a, b) <= 1e-12   # the same per-electron contributions, summed in FP64


def test_fp64_follows_algorithm_2_step_by_step_when_a_step_is_superluminal():
    """A sampled step longer than c0 dt (the advanced time can decrease for some
    directions): the upload flags LW_ST_STEP and the FP64 deposit follows Algorithm 2
    step by step, repeated grid points and LW_ST_TA_ORDER included, like the oracle."""
    tr = simple.random_smooth(3, 120, 2e-18, 17, gamma=6.0, amp=0.4)
    r = tr.r.copy()
    r[1, 60:, 2] += 3.0 * 299792458.0 * 2e-18     # a jump of 3 c0 dt between two samples
    bad = simple.Trajectories(tr.t, r, tr.beta, tr.beta_dot)
    n_hat = np.array([[0.0, 0.0, 1.0], [0.05, 0.0, math.sqrt(1 - 0.0025)]])
    lo, hi = oracle.grid_bounds(bad.t, bad.r, n_hat)
    grid = lw.Grid(lo, (hi - lo) / 200, 256)
    g = gpu_run(bad, n_hat, grid, lw.LW_FP64, spectrum=False)
    o = oracle_run(bad, n_hat, grid, spectrum=False)
    assert g["status"] & lw.LW_ST_STEP
    assert o["status"] & oracle.ST_TA_ORDER
    assert (g["status"] & ~lw.LW_ST_STEP) == o["status"]
    assert np.max(np.abs(g["rec"] - o["rec"])) <= 1e-12 * np.abs(o["rec"]).max()


@pytest.mark.parametrize("block", [16, 512])
def test_mixed_section_values(block):
    """The upload's mixed section: per sample (tau - tau_b, r - r_b) rounded to FP32 from
    FP64 differences, and (beta_x, beta_y, 1 - beta_z, beta_dot) rounded to FP32 --
    bit-exact against numpy's round-to-nearest casts (tau to one FP64 rounding, as the
    device may fuse the light-front product)."""
    tr = simple.random_smooth(5, 700, 2e-18, 23, gamma=30.0, amp=0.3, t_per_electron=True)
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot, block=block)
    scan, field = [x.cpu().numpy() for x in traj.mixed_section()]
    ib = (np.arange(tr.n_s + 1) // block) * block
    rb = tr.r[:, ib, :]
    for c in range(3):
        assert np.array_equal(scan[..., 1 + c], (tr.r[..., c] - rb[..., c]).astype(np.float32))
    tau = tr.t - tr.r[..., 2] / 299792458.0
    dtau = tau - tau[:, ib]
    assert np.all(np.abs(scan[..., 0] - dtau) <= 4e-16 * np.abs(tau) + 1e-7 * np.abs(dtau))
    assert np.array_equal(field[..., 0], tr.beta[..., 0].astype(np.float32))
    assert np.array_equal(field[..., 1], tr.beta[..., 1].astype(np.float32))
    assert np.array_equal(field[..., 2:4], tr.beta_dot[..., :2].astype(np.float32))
    assert np.array_equal(field[..., 4], (1.0 - tr.beta[..., 2]).astype(np.float32))
    assert np.array_equal(field[..., 5], tr.beta_dot[..., 2].astype(np.float32))


def test_config3_mixed_spectrum_per_band():
    """Config 3 (the mixed path on config 1's inputs): spectrum relative L2 error against
    the FP64 oracle in the band of the Doppler fundamental omega_1(theta) +-20 % of every
    pixel (<= 1e-4) and in the 2nd-harmonic band, where the on-axis line is weak for
    linear polarisation and the relative error is expected to be larger (<= 1e-2)."""
    from workloads.planewave import doppler_fundamental
    w = configs.c1_tiny()
    tr = w.traj
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot)
    det = lw.Detector(w.n_hat)
    b = lw.lw_grid_bounds(traj, det).cpu().numpy()
    grid = lw.grid_from_bounds(b[0], b[1], w.n_bins)
    S = lw.lw_spectrum(lw.lw_deposit_time_domain(traj, det, grid, lw.LW_MIXED), lw.LW_MIXED,
                       det.n_pix, grid).double().cpu().numpy()
    rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, w.n_hat, grid.t_min,
                                grid.dt_u, grid.n_bins)
    S_o = oracle.spectrum(rec, grid.dt_u)
    omega = 2 * math.pi * np.arange(grid.n_bins // 2 + 1) / (grid.n_bins * grid.dt_u)
    theta = np.arccos(np.clip(w.n_hat[:, 2], -1.0, 1.0))
    w1 = np.array([doppler_fundamental(w.gamma, w.lam, w.a0, th) for th in theta])
    for h, tol in ((1.0, 1e-4), (2.0, 1e-2)):
        band = np.abs(omega[None, :] / (h * w1[:, None]) - 1.0) <= 0.2
        assert band.sum() > w.n_pix
        err = np.linalg.norm((S - S_o)[band]) / np.linalg.norm(S_o[band])
        assert err <= tol, (h, err)


def test_precision_bit_flags_a_coarsely_sampled_synchrotron_flash():
    """LW_ST_PRECISION: an observer in the orbit plane of electrons circling at beta = 0.999,
    sampled 100 times per turn, sees a flash that changes by a large fraction across a
    step; the mixed deposit's FP32 weights and Doppler factors err by more than 1e-4 of
    the spectrum (checked against the oracle) and every mixed record reports it.  The FP64
    path matches the oracle and reports nothing."""
    dt = 1e-16
    tr = simple.circular_motion(4096, dt, 0.999, 2 * math.pi / (100 * dt), n_e=4)
    ang = np.linspace(-0.02, 0.02, 4)
    n_hat = np.stack([np.cos(ang), np.zeros_like(ang), np.sin(ang)], -1)
    lo, hi = oracle.grid_bounds(tr.t, tr.r, n_hat)
    grid = lw.grid_from_bounds(lo, hi, 8192)
    o = oracle_run(tr, n_hat, grid)
    g64 = gpu_run(tr, n_hat, grid, lw.LW_FP64, block=512)
    assert g64["status"] & lw.LW_ST_PRECISION == 0
    assert rel_l2(g64["S"], o["S"]) <= FP64_TOL
    for prec in (lw.LW_MIXED, lw.LW_MIXED_KAHAN, lw.LW_MIXED_F32, lw.LW_MIXED_F32X4):
        g = gpu_run(tr, n_hat, grid, prec, block=512)
        assert rel_l2(g["S"], o["S"]) > MIXED_TOL
        assert g["status"] & lw.LW_ST_PRECISION, prec


def test_precision_bit_quiet_on_a_resolved_bunch():
    """No LW_ST_PRECISION on a Boris-pushed bunch in the laser (300 electrons, 3,000 steps,
    32 x 32 pixels, 65,536 bins), whose mixed spectrum is within 1e-4 of the FP64 one."""
    w = configs.c2_paper(n_e=300, n_s=3000, nx=32)
    tr = w.traj
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot)
    det = lw.Detector(w.n_hat)
    b = lw.lw_grid_bounds(traj, det).cpu().numpy()
    grid = lw.grid_from_bounds(b[0], b[1], w.n_bins)
    S64 = lw.lw_spectrum(lw.lw_deposit_time_domain(traj, det, grid, lw.LW_FP64), lw.LW_FP64,
                         det.n_pix, grid)
    for prec in (lw.LW_MIXED, lw.LW_MIXED_F32X4):
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        S = lw.lw_spectrum(lw.lw_deposit_time_domain(traj, det, grid, prec, status=st), prec,
                           det.n_pix, grid)
        torch.cuda.synchronize()
        assert int(st.item()) & lw.LW_ST_PRECISION == 0
        assert float(torch.linalg.norm(S.double() - S64) / torch.linalg.norm(S64)) <= MIXED_TOL


def test_precision_check_launch_leaves_the_record_complete():
    """With a status word the deposit launches its precision check as a programmatic
    dependent (it starts beside the deposit's last CTAs and ends only after the deposit
    grid); a spectrum enqueued right after must see the finished record: records and
    spectra equal those of a deposit without the check, up to the order of the FP32
    reductions, on a case with enough electron chunks for the check's stride of 64."""
    w = configs.c2_paper(n_e=400, n_s=2000, nx=32, n_bins=16384)
    tr = w.traj
    dev = torch.device("cuda")
    traj = lw.lw_trajectories_upload(tr.t, tr.r, tr.beta, tr.beta_dot,
                                     sections=lw.LW_SECTION_MIXED, device=dev)
    det = lw.Detector(w.n_hat, device=dev)
    b = lw.lw_grid_bounds(traj, det).cpu().numpy()
    grid = lw.grid_from_bounds(b[0], b[1], w.n_bins)
    P = lw.LW_MIXED_F32X4
    rec_a = lw.lw_deposit_time_domain(traj, det, grid, P)
    S_a = lw.lw_spectrum(rec_a, P, det.n_pix, grid)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rec_b = lw.lw_deposit_time_domain(traj, det, grid, P, status=status)
    S_b = lw.lw_spectrum(rec_b, P, det.n_pix, grid)
    torch.cuda.synchronize()
    ra, rb = rec_a.double().cpu().numpy(), rec_b.double().cpu().numpy()
    assert np.abs(ra).max() > 0
    assert rel_l2(rb, ra) <= 1e-6
    assert rel_l2(S_b.double().cpu().numpy(), S_a.double().cpu().numpy()) <= 1e-6
