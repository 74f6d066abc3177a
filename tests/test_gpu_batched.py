"""Batched persistent deposit (several variants, one launch): equal to the
per-variant deposit, autotuned tile shapes, CUDA-graph replay, and the FP64
oracle on sampled variants and pixels."""
import numpy as np
import pytest
import torch

import oracle
from gpu_cases import rel_l2
from paper_2206_03015_gb300 import lw
from paper_2206_03015_gb300.autotune import Autotuner
from workloads import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def variants():
    vs = configs.c5_batch(n_variants=7, n_e=(12, 48), n_s=(2500, 5000), nx=(4, 12),
                          log2_bins=(10, 13))
    out = []
    for v in vs:
        w = v.build()
        tr = w.traj
        inputs = tuple(torch.from_numpy(x).cuda() for x in (tr.t, tr.r, tr.beta, tr.beta_dot))
        traj = lw.lw_trajectories_upload(*inputs, sections=lw.LW_SECTION_MIXED)
        det = lw.Detector(w.n_hat)
        b = lw.lw_grid_bounds(traj, det).cpu().numpy()
        grid = lw.grid_from_bounds(b[0], b[1], w.n_bins)
        out.append((w, inputs, traj, det, grid))
    return out


def _records(variants, precision=lw.LW_MIXED):
    recs = []
    for (_, _, _, det, grid) in variants:
        shp, dt = lw.record_shape(det, grid, precision)
        recs.append(torch.empty(shp, dtype=dt, device="cuda"))
    return recs


@pytest.mark.parametrize("precision,tol", [(lw.LW_MIXED, 1e-12), (lw.LW_MIXED_F32, 1e-6),
                                           (lw.LW_MIXED_F32X4, 1e-6)])
def test_batched_equals_per_variant(variants, precision, tol):
    recs = _records(variants, precision)
    bp = lw.lw_batch_plan([v[2] for v in variants], [v[3] for v in variants],
                          [v[4] for v in variants], recs, precision=precision)
    assert bp.plan.n_units >= len(variants)
    lw.lw_batch_deposit(bp)
    for (w, _, traj, det, grid), rec in zip(variants, recs):
        ref = lw.lw_deposit_time_domain(traj, det, grid, precision)
        torch.cuda.synchronize()
        # FP32 records: the same contributions, added in another order
        assert rel_l2(rec.double().cpu().numpy(), ref.double().cpu().numpy()) <= tol, w.name


def test_autotuned_batch_matches_oracle_on_sampled_variants(variants):
    tuner = Autotuner(reps=1)
    trajs, chunks = [], []
    for (_, inputs, _, det, grid) in variants:
        c = tuner.tune(inputs, det, grid, blocks=(64, 128), chunks=(1, 4, 16))
        trajs.append(lw.lw_trajectories_upload(*inputs, sections=lw.LW_SECTION_MIXED,
                                               block=c.block))
        chunks.append(c.e_chunk)
    recs = _records(variants)
    bp = lw.lw_batch_plan(trajs, [v[3] for v in variants], [v[4] for v in variants], recs,
                          e_chunks=chunks)
    lw.lw_batch_deposit(bp)
    for idx in (0, 2, 4, len(variants) - 1):   # four sampled variants
        w, _, _, det, grid = variants[idx]
        S = lw.lw_spectrum(recs[idx], lw.LW_MIXED, det.n_pix, grid).double().cpu().numpy()
        pix = np.arange(0, w.n_pix, max(1, w.n_pix // 5))
        tr = w.traj
        ref, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, w.n_hat[pix], grid.t_min,
                                    grid.dt_u, grid.n_bins)
        S_o = oracle.spectrum(ref, grid.dt_u)
        assert rel_l2(S[pix], S_o) <= 1e-4, w.name


def test_batch_and_spectra_replay_from_a_cuda_graph(variants):
    recs = _records(variants)
    bp = lw.lw_batch_plan([v[2] for v in variants], [v[3] for v in variants],
                          [v[4] for v in variants], recs)
    outs = [torch.empty((v[3].n_pix, v[4].n_bins // 2 + 1), dtype=torch.float32, device="cuda")
            for v in variants]
    wss = [lw.workspace(lw.spectrum_workspace_bytes(lw.LW_MIXED, v[3].n_pix, v[4]))
           for v in variants]

    def run():
        lw.lw_batch_deposit(bp)
        for v, rec, o, ws in zip(variants, recs, outs, wss):
            lw.lw_spectrum(rec, lw.LW_MIXED, v[3].n_pix, v[4], ws=ws, out=o)

    run()                                  # eager, also sets kernel attributes
    torch.cuda.synchronize()
    eager = [o.clone() for o in outs]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            run()
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        for o, e in zip(outs, eager):
            assert rel_l2(o.double().cpu().numpy(), e.double().cpu().numpy()) <= 1e-5
