"""lw_spectrum_static -- the spectrum entry point that allocates nothing and
uses the library's fixed device scratch array -- gives the same spectra as
lw_spectrum with a caller-supplied workspace, on two calls in a row (the
array keeps the previous call's contents), for the single-pass and the
four-step transform and for both record precisions.  Runs last so that a
failure here does not hide any other test."""
import math

import numpy as np
import pytest
import torch

from paper_2206_03015_gb300 import lw

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


@pytest.mark.parametrize("n_bins,n_pix", [(4096, 64), (8192, 5), (65536, 7)])
@pytest.mark.parametrize("precision", [lw.LW_FP64, lw.LW_MIXED, lw.LW_MIXED_KAHAN,
                                       lw.LW_MIXED_F32])
def test_static_scratch_matches_workspace_entry_point(n_bins, n_pix, precision):
    grid = lw.Grid(0.0, 2.9e-18, n_bins)
    tol = 1e-12 if precision == lw.LW_FP64 else 1e-5
    for call in range(2):
        rng = np.random.Generator(np.random.PCG64(1000 * call + n_bins + n_pix + precision))
        rec = rng.normal(size=(n_pix, 3, n_bins)) * 1e20
        if precision == lw.LW_MIXED_KAHAN:
            hi = rec.astype(np.float32)
            lo = (rec - hi.astype(np.float64)).astype(np.float32)
            r = torch.from_numpy(np.stack([hi, lo], -1)).cuda()
        elif precision == lw.LW_MIXED_F32:
            r = torch.from_numpy(rec.astype(np.float32)).cuda()
        else:
            r = torch.from_numpy(rec).cuda()
        S_ref, X_ref = lw.lw_spectrum(r, precision, n_pix, grid, want_X=True)
        S, X = lw.lw_spectrum_static(r, precision, n_pix, grid, want_X=True)
        torch.cuda.synchronize()
        assert _rel(S, S_ref) <= tol, (call, _rel(S, S_ref))
        assert _rel(torch.view_as_real(X), torch.view_as_real(X_ref)) <= tol


def test_static_scratch_rejects_oversized_transforms():
    lib = lw.load()
    cap = lib.lw_spectrum_static_capacity()
    n_bins = 1 << 17
    n_pix = 2 * math.ceil(cap / (3 * n_bins * 16)) + 2     # FP64 four-step needs more than cap
    grid = lw.Grid(0.0, 1e-18, n_bins)
    rec = torch.zeros((n_pix, 3, n_bins), dtype=torch.float64, device="cuda")
    with pytest.raises(lw.LWError) as e:
        lw.lw_spectrum_static(rec, lw.LW_FP64, n_pix, grid)
    assert e.value.code == lw.LW_ESIZE
