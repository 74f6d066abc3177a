"""On the GPU: device tensors of the wrong type, layout or size are refused by the binding
before the library is called (no kernel runs on them)."""
import pytest
import torch

from paper_2206_03015_gb300 import lw

pytestmark = pytest.mark.gpu


def test_device_tensors_of_wrong_type_or_size_are_refused():
    n_pix, n_bins = 4, 256
    grid = lw.Grid(0.0, 1e-18, n_bins)
    nl = n_bins // 2 + 1
    rec64 = torch.zeros((n_pix, 3, n_bins), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError, match="record: torch.float32 given"):
        lw.lw_spectrum(rec64.float(), lw.LW_FP64, n_pix, grid)
    with pytest.raises(ValueError, match="record: .* elements given"):
        lw.lw_spectrum(rec64[:n_pix - 1], lw.LW_FP64, n_pix, grid)
    with pytest.raises(ValueError, match="record: a contiguous tensor"):
        lw.lw_spectrum(rec64.transpose(1, 2), lw.LW_FP64, n_pix, grid)
    with pytest.raises(ValueError, match="out: .* elements given"):
        lw.lw_spectrum(rec64, lw.LW_FP64, n_pix, grid,
                       out=torch.empty((n_pix - 1, nl), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError, match="out: torch.float32 given"):
        lw.lw_spectrum_static(rec64, lw.LW_FP64, n_pix, grid,
                              out=torch.empty((n_pix, nl), dtype=torch.float32, device="cuda"))
    ws = lw.workspace(1 << 20)
    with pytest.raises(ValueError, match="256-byte boundary"):
        lw.lw_spectrum(rec64, lw.LW_FP64, n_pix, grid, ws=ws[8:])
    n_e, n_s = 2, 8
    r = torch.zeros((n_e, 3), dtype=torch.float64, device="cuda")
    t = torch.empty(n_s, dtype=torch.float64, device="cuda")           # one too few
    outs = [torch.empty((n_e, n_s + 1, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(ValueError, match="t_out: 8 elements given, at least 9"):
        lw.lw_boris_push(r, r.clone(), 0.0, 1e-17, n_s, (0.8e-6, 0.5, 20e-6, 30e-15), t, *outs)
