"""Host-side logic of the benchmark: the profile source key, the clock-record parser and
the grid-point count used for the atomic rate (no GPU needed)."""
import importlib.util
import math
import os

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_source_key_ignores_comments_and_layout_but_not_code(tmp_path):
    b = _bench()
    a = tmp_path / "a.cu"
    a.write_text("// header\n__global__ void k(int* p) {\n  p[0] = 1;  /* set */\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("/* another\n   header */\n__global__   void k(int* p)\n{ p[0] = 1; // set\n}\n")
    d = tmp_path / "d.cu"
    d.write_text("__global__ void k(int* p) { p[0] = 2; }\n")
    assert b._source_hash(str(a)) == b._source_hash(str(c))
    assert b._source_hash(str(a)) != b._source_hash(str(d))


def test_clock_record_parser_takes_median_and_active_reasons():
    b = _bench()
    s = b.ClockSampler(0)

    class _P:   # stands in for the nvidia-smi process whose output lines are parsed
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc = _P()
    s.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbled line",
    ]
    out = s.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_grid_points_reached_counts_the_exact_end_bins():
    """Per (pixel, electron): the points of (floor(u_first), floor(u_last)] in [0, n_bins),
    recounted here by brute force over the grid points."""
    b = _bench()
    from paper_2206_03015_gb300 import lw
    rng = np.random.Generator(np.random.PCG64(7))
    n_e, ns1, n_pix, n_bins = 5, 9, 4, 40
    c0 = 299792458.0
    t = np.sort(rng.uniform(0, 1e-15, ns1))
    r = rng.normal(scale=1e-7, size=(n_e, ns1, 3))
    th = rng.uniform(-0.05, 0.05, (n_pix, 2))
    n_hat = np.stack([np.sin(th[:, 0]), np.cos(th[:, 0]) * np.sin(th[:, 1]),
                      np.cos(th[:, 0]) * np.cos(th[:, 1])], -1)
    ta0 = t[0] - (r[:, 0, :] @ n_hat.T).T / c0      # [pix][e]
    ta1 = t[-1] - (r[:, -1, :] @ n_hat.T).T / c0
    t_min = float(ta0.min()) + 2e-17   # some first samples fall before the grid
    dt_u = float(ta1.max() - ta0.min()) / (n_bins - 5)
    grid = lw.Grid(t_min, dt_u, n_bins)

    class _Det:
        pass

    det = _Det()
    det.n_pix = n_pix
    det.n_hat = torch.from_numpy(n_hat)
    got = b.grid_points_reached(torch.from_numpy(t), torch.from_numpy(r), det, grid)
    want = 0
    for m in range(n_pix):
        for k in range(n_e):
            u0 = (ta0[m, k] - t_min) / dt_u
            u1 = (ta1[m, k] - t_min) / dt_u
            want += sum(1 for j in range(n_bins) if math.floor(u0) < j <= math.floor(u1))
    assert got == want


def test_deposit_roofline_picks_the_binding_pipe():
    """The work model and the bound with the largest fraction of its measured peak."""
    b = _bench()
    from paper_2206_03015_gb300 import lw
    w = b.deposit_work(10_000, 10_000, 4096, 65_536, 512, 885_159_358, lw.LW_MIXED_F32X4)
    assert w["pixel_blocks"] == 4096 * 10_000 * 20     # 10,000 steps in blocks of 512
    assert w["l2_ops"] == 885_159_358
    assert w["hbm_bytes"] == 10_000 * (10_001 * 40 + 20 * 32) + 4096 * 3 * 65_536 * 4
    assert w["fp32_flops"] == 885_159_358 * 86 + 4096 * 10_000 * 20 * 47
    w3 = b.deposit_work(10_000, 10_000, 4096, 65_536, 512, 100, lw.LW_MIXED)
    assert w3["l2_ops"] == 300 and w3["hbm_bytes"] > w["hbm_bytes"]
    peaks = {"red_v4f32_lines": {"ops_per_s": 2.0e11}, "fma_f32": {"flops": 75e12},
             "lds_v4": {"bytes_per_s": 40e12}}
    r = b.deposit_roofline(w, 10.0, peaks, 6800.0)
    t = 10e-3
    assert r["bound"] == "l2_red"
    assert math.isclose(r["achieved"], 885_159_358 / t / 1e9)
    assert math.isclose(r["frac"], 885_159_358 / t / 2.0e11)
    for k, v in r["bounds"].items():
        assert v["frac"] <= r["frac"] and math.isclose(v["frac"], v["achieved"] / v["peak"])
