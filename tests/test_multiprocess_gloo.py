"""Detector and beam parallelization across processes (world size 2, gloo, CPU):
both reproduce the single-process record and spectrum.  The per-rank work is
done by the CPU oracle here; the GPU path is one process per GPU with the same
host-side decomposition."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2206_03015_gb300 import parallel


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    from workloads import simple
    tr = simple.random_smooth(5, 120, 2e-18, 77, gamma=5.0, amp=0.5)
    rng = np.random.Generator(np.random.PCG64(3))
    tx, ty = rng.uniform(-0.2, 0.2, 7), rng.uniform(-0.2, 0.2, 7)
    n_hat = np.stack([np.sin(tx), np.cos(tx) * np.sin(ty), np.cos(tx) * np.cos(ty)], -1)
    return tr, n_hat


def _worker(rank, world, port, scheme, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        tr, n_hat = _case()
        lo_t, hi_t = oracle.grid_bounds(tr.t, tr.r, n_hat)
        n_bins = 256
        dt_u = (hi_t - lo_t) / n_bins
        if scheme == "detector":
            lo, hi = parallel.pixel_shard(n_hat.shape[0], rank, world)
            rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat[lo:hi], lo_t,
                                        dt_u, n_bins)
            S = torch.from_numpy(oracle.spectrum(rec, dt_u)) if hi > lo else \
                torch.zeros((0, n_bins // 2 + 1), dtype=torch.float64)
            S_all = parallel.gather_pixels(S, dist)
            rec_all = parallel.gather_pixels(torch.from_numpy(rec), dist)
        else:
            lo, hi = parallel.beam_shard(tr.n_e, rank, world)
            sub = tr.subset(slice(lo, hi))
            rec, _ = oracle.tdm_deposit(sub.t, sub.r, sub.beta, sub.beta_dot, n_hat, lo_t, dt_u,
                                        n_bins)
            rec_all = parallel.reduce_beam(torch.from_numpy(rec), dist)
            S_all = torch.from_numpy(oracle.spectrum(rec_all.numpy(), dt_u))
        if rank == 0:
            torch.save({"rec": rec_all, "S": S_all}, out_path)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("scheme", ["detector", "beam"])
def test_two_process_decomposition_matches_single_process(scheme, tmp_path):
    import oracle
    out = str(tmp_path / f"{scheme}.pt")
    mp.start_processes(_worker, args=(2, _free_port(), scheme, out), nprocs=2, join=True,
                       start_method="spawn")
    got = torch.load(out)
    tr, n_hat = _case()
    lo_t, hi_t = oracle.grid_bounds(tr.t, tr.r, n_hat)
    dt_u = (hi_t - lo_t) / 256
    rec, _ = oracle.tdm_deposit(tr.t, tr.r, tr.beta, tr.beta_dot, n_hat, lo_t, dt_u, 256)
    S = oracle.spectrum(rec, dt_u)
    tol = 0.0 if scheme == "detector" else 1e-12
    assert np.max(np.abs(got["rec"].numpy() - rec)) <= tol * np.abs(rec).max()
    assert np.max(np.abs(got["S"].numpy() - S)) <= max(tol, 1e-12) * np.abs(S).max()


def test_shards_partition_and_scheme_choice():
    for n in (0, 1, 7, 4096):
        for world in (1, 2, 3, 8):
            rs = [parallel.balanced_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [h - l for l, h in rs]
            assert max(sizes) - min(sizes) <= 1
    # Eq. (parallel_scheme_function_2) and the memory model agree
    for N_p, N_obs, N_Tu in ((6.25e6, 4096, 65536), (1e7, 10, 1000), (1e4, 4096, 65536)):
        pref = parallel.preferred_scheme(N_p, N_obs, N_Tu)
        mb = parallel.memory_per_rank("beam", 8, N_p, N_obs, N_Tu)
        md = parallel.memory_per_rank("detector", 8, N_p, N_obs, N_Tu)
        assert (pref == "detector") == (md <= mb)


def _bench_module():
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_shard", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _bench_worker(rank, world, port, out_path):
    """What bench.py does per rank under torchrun, without a GPU: its pixel block of the
    one detector, its deposits, and the MAX over ranks of its step time."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench_module()
        n_e, n_s, n_pix = 10_000, 10_000, 4096
        lo, hi = b.shard_pixels(n_pix, rank, world)
        mine = torch.tensor([lo, hi, n_e * n_s * (hi - lo)], dtype=torch.int64)
        got = [torch.zeros(3, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(got, mine)
        ms = torch.tensor([10.0 + rank], dtype=torch.float64)
        dist.all_reduce(ms, op=dist.ReduceOp.MAX)
        if rank == 0:
            torch.save({"shards": torch.stack(got), "ms": float(ms.item()),
                        "job": b.job_deposits(n_e, n_s, n_pix, world)}, out_path)
    finally:
        dist.destroy_process_group()


def test_bench_pixel_shards_cover_one_detector(tmp_path):
    """bench.py --gpus 2: the two ranks' pixel blocks partition the detector, their
    deposits add up to the job's, and the step time is the slower rank's."""
    out = str(tmp_path / "bench.pt")
    mp.start_processes(_bench_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    got = torch.load(out)
    sh = got["shards"].numpy()
    assert sh[0][0] == 0 and sh[0][1] == sh[1][0] and sh[1][1] == 4096
    assert int(sh[:, 2].sum()) == got["job"] == 10_000 * 10_000 * 4096
    assert got["ms"] == 11.0
    b = _bench_module()
    assert b.shard_pixels(4096, 1, 2, "detectors") == (0, 4096)
    assert b.job_deposits(10, 10, 4, 2, "detectors") == 800
