"""Tile-shape autotuner for the batched (persistent) mixed deposit.

For each variant the tuner times the persistent kernel on that variant alone
for every (samples per anchoring block, electrons per work unit) pair in a
small candidate set and keeps the fastest.  Results are cached per problem
shape (in memory and, optionally, in a JSON file) so a repeated sweep does not
re-tune.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import torch

from . import lw

BLOCKS = (128, 256, 512)
CHUNKS = (1, 2, 4, 8, 16, 32)


@dataclass
class Choice:
    block: int
    e_chunk: int
    ms: float


def shape_key(n_e, n_s, n_pix, n_bins):
    return f"{n_e}x{n_s}x{n_pix}x{n_bins}"


class Autotuner:
    def __init__(self, cache_path: str | None = None, reps: int = 2):
        self.cache_path = cache_path
        self.reps = reps
        self.cache: dict[str, dict] = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def save(self):
        if self.cache_path:
            tmp = self.cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.cache_path)

    def _time(self, traj, det, grid, record, e_chunk, precision=lw.LW_MIXED):
        bp = lw.lw_batch_plan([traj], [det], [grid], [record], precision=precision,
                              e_chunks=[e_chunk])
        lw.lw_batch_deposit(bp)                       # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(self.reps):
            lw.lw_batch_deposit(bp)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / self.reps

    def tune(self, inputs, det, grid, blocks=BLOCKS, chunks=CHUNKS,
             precision=lw.LW_MIXED) -> Choice:
        """inputs: (t, r, beta, beta_dot) device tensors of one variant; precision: the
        mixed record the batch will use."""
        n_e, ns1, _ = inputs[1].shape
        key = shape_key(n_e, ns1 - 1, det.n_pix, grid.n_bins) + f"/{precision}"
        if key in self.cache:
            c = self.cache[key]
            return Choice(c["block"], c["e_chunk"], c["ms"])
        shp, dt = lw.record_shape(det, grid, precision)
        record = torch.empty(shp, dtype=dt, device=det.n_hat.device)
        best = None
        for block in blocks:
            traj = lw.lw_trajectories_upload(*inputs, sections=lw.LW_SECTION_MIXED, block=block,
                                             device=det.n_hat.device)
            for ch in chunks:
                if ch > n_e:
                    continue
                ms = self._time(traj, det, grid, record, ch, precision)
                if best is None or ms < best.ms:
                    best = Choice(block, ch, ms)
        self.cache[key] = {"block": best.block, "e_chunk": best.e_chunk, "ms": best.ms}
        return best
