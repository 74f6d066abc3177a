"""The autotuner's host logic without a GPU: a choice is cached under the variant's
shape and record type, written to its JSON file atomically, read back by a new tuner,
and a cached shape is answered without timing anything."""
import json
from types import SimpleNamespace

import torch

from paper_2206_03015_gb300 import autotune, lw


def test_cached_choice_round_trips_through_the_file(tmp_path):
    path = str(tmp_path / "tune.json")
    n_e, n_s, n_pix, n_bins = 64, 2000, 256, 4096
    key = autotune.shape_key(n_e, n_s, n_pix, n_bins) + f"/{lw.LW_MIXED_F32X4}"
    t = autotune.Autotuner(path)
    t.cache[key] = {"block": 256, "e_chunk": 4, "ms": 1.25}
    t.save()
    assert json.load(open(path)) == {key: {"block": 256, "e_chunk": 4, "ms": 1.25}}

    # a fresh tuner answers from the file; the inputs are CPU tensors and nothing is timed
    t2 = autotune.Autotuner(path)
    inputs = (torch.zeros(n_s + 1), torch.zeros(n_e, n_s + 1, 3),
              torch.zeros(n_e, n_s + 1, 3), torch.zeros(n_e, n_s + 1, 3))
    det = SimpleNamespace(n_pix=n_pix)
    grid = SimpleNamespace(n_bins=n_bins)
    c = t2.tune(inputs, det, grid, precision=lw.LW_MIXED_F32X4)
    assert (c.block, c.e_chunk, c.ms) == (256, 4, 1.25)


def test_shape_key_separates_shapes():
    keys = {autotune.shape_key(*s) for s in [(1, 2, 3, 4), (2, 1, 3, 4), (1, 2, 4, 3)]}
    assert len(keys) == 3
