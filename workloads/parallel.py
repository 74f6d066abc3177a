"""Parallel generation of large Boris-pushed bunches.

Electrons are independent, so the bunch is split into fixed chunks of
``CHUNK`` electrons (the split does not depend on the number of workers, so
the bytes are identical for any worker count) and pushed in a ``spawn``
process pool that writes straight into shared memory.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from .boris import GaussianLaser, boris_trajectories
from .simple import Trajectories

CHUNK = 256


def _worker(args):
    (names, shape, r0, u0, laser, t_start, t_end, n_steps, lo, hi) = args
    shms = [shared_memory.SharedMemory(name=n) for n in names]
    try:
        R, B, D = (np.ndarray(shape, dtype=np.float64, buffer=s.buf) for s in shms)
        tr = boris_trajectories(r0, u0, laser, t_start, t_end, n_steps)
        R[lo:hi] = tr.r
        B[lo:hi] = tr.beta
        D[lo:hi] = tr.beta_dot
    finally:
        for s in shms:
            s.close()
    return hi - lo


def boris_trajectories_parallel(r0, u0, laser: GaussianLaser, t_start: float, t_end: float,
                                n_steps: int, workers: int | None = None) -> Trajectories:
    n_e = r0.shape[0]
    if workers is None:
        workers = max(1, min(os.cpu_count() or 1, 16))
    if n_e <= CHUNK:
        return boris_trajectories(r0, u0, laser, t_start, t_end, n_steps)
    shape = (n_e, n_steps + 1, 3)
    nbytes = int(np.prod(shape)) * 8
    shms = [shared_memory.SharedMemory(create=True, size=nbytes) for _ in range(3)]
    try:
        jobs = []
        for lo in range(0, n_e, CHUNK):
            hi = min(n_e, lo + CHUNK)
            jobs.append(([s.name for s in shms], shape, r0[lo:hi], u0[lo:hi], laser, t_start,
                         t_end, n_steps, lo, hi))
        if workers == 1:
            done = sum(_worker(j) for j in jobs)
        else:
            ctx = mp.get_context("spawn")
            with ctx.Pool(workers) as pool:
                done = sum(pool.map(_worker, jobs, chunksize=1))
        assert done == n_e
        out = [np.ndarray(shape, dtype=np.float64, buffer=s.buf).copy() for s in shms]
    finally:
        for s in shms:
            s.close()
            s.unlink()
    dt = (t_end - t_start) / n_steps
    t = t_start + dt * np.arange(n_steps + 1)
    return Trajectories(t, out[0], out[1], out[2])
