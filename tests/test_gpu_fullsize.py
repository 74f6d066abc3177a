"""C2 at full size (10,000 electrons x 10,000 Boris steps x 64x64 pixels, 65,536 bins) in
the launch configuration the benchmark times: device-resident FP64 inputs, anchoring
block 512, grid from the device bounds (Eqs. tu_min, tu_max), spectrum by the four-step
passes.  Sampled pixels are checked against the CPU oracle run for those pixels alone;
over all pixels, the mixed spectrum is checked against the FP64 path.

Tolerances as in the small parity cases: FP64 1e-9 relative L2 (contributions are
bit-identical, only the summation order differs), mixed 1e-4 on spectra."""
import numpy as np
import pytest
import torch

import oracle
from gpu_cases import rel_l2
from paper_2206_03015_gb300 import lw
from workloads import configs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
MIXED_TOL = 1e-4
# corners, the axis and two off-axis pixels of the 64 x 64 detector
SAMPLE = [0, 63, 2080, 1000, 3333, 4095]
# every precision: FP64, and the mixed path with each of its records (FP64, compensated FP32
# pairs, plain FP32, FP32 interleaved per grid point -- the last is the one the benchmark
# times)
MODES = {"fp64": lw.LW_FP64, "mixed": lw.LW_MIXED, "mixed_kahan": lw.LW_MIXED_KAHAN,
         "mixed_f32": lw.LW_MIXED_F32, "mixed_f32x4": lw.LW_MIXED_F32X4}
MIXED = ["mixed", "mixed_kahan", "mixed_f32", "mixed_f32x4"]


@pytest.fixture(scope="module")
def c2():
    w = configs.c2_paper()
    tr = w.traj
    dev = torch.device("cuda")
    t_d, r_d, b_d, a_d = (torch.from_numpy(x).to(dev)
                          for x in (tr.t, tr.r, tr.beta, tr.beta_dot))
    det = lw.Detector(w.n_hat, device=dev)
    traj = lw.lw_trajectories_upload(t_d, r_d, b_d, a_d,
                                     sections=lw.LW_SECTION_FP64 | lw.LW_SECTION_MIXED,
                                     block=512, device=dev)
    b = lw.lw_grid_bounds(traj, det).cpu().numpy()
    grid = lw.grid_from_bounds(b[0], b[1], w.n_bins)
    out = {"w": w, "grid": grid}
    for name, prec in MODES.items():
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        rec = lw.lw_deposit_time_domain(traj, det, grid, prec, status=status)
        S = lw.lw_spectrum(rec, prec, det.n_pix, grid)
        val = lw.record_value(rec, prec)
        out[name] = {"rec": val[SAMPLE].double().cpu().numpy(), "S": S.double(),
                     "status": int(status.item())}
        del rec, val
    rec_o, st_o = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, w.n_hat[SAMPLE],
                                     grid.t_min, grid.dt_u, grid.n_bins)
    out["oracle"] = {"rec": rec_o, "S": oracle.spectrum(rec_o, grid.dt_u), "status": st_o}
    torch.cuda.synchronize()
    return out


def test_c2_fp64_sampled_pixels_match_oracle(c2):
    g, o = c2["fp64"], c2["oracle"]
    assert o["status"] & ~g["status"] == 0   # the sampled pixels' bits (the GPU's cover all)
    for k, m in enumerate(SAMPLE):
        assert np.array_equal(g["rec"][k] != 0, o["rec"][k] != 0), m   # same bins reached
        assert rel_l2(g["rec"][k], o["rec"][k]) <= FP64_TOL, m
        assert rel_l2(g["S"][m].cpu().numpy(), o["S"][k]) <= FP64_TOL, m


@pytest.mark.parametrize("mode", MIXED)
def test_c2_mixed_sampled_pixels_match_oracle(c2, mode):
    g, o = c2[mode], c2["oracle"]
    assert o["status"] & ~g["status"] == 0
    for k, m in enumerate(SAMPLE):
        assert rel_l2(g["S"][m].cpu().numpy(), o["S"][k]) <= MIXED_TOL, m
        # the record itself, element-wise against the oracle's largest value
        scale = np.abs(o["rec"][k]).max()
        assert np.abs(g["rec"][k] - o["rec"][k]).max() <= MIXED_TOL * scale, m


@pytest.mark.parametrize("mode", MIXED)
def test_c2_mixed_matches_fp64_over_all_pixels(c2, mode):
    a, b = c2[mode]["S"], c2["fp64"]["S"]
    err = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    assert err <= MIXED_TOL, err
    # per pixel as well: no pixel's spectrum is off by more than the tolerance
    per = torch.linalg.norm(a - b, dim=1) / torch.linalg.norm(b, dim=1)
    assert float(per.max()) <= MIXED_TOL, float(per.max())
