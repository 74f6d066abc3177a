"""The binding refuses tensors that the library would read or write as device memory when
they are not device memory of the right type and size: a host tensor, a wrong dtype, a
non-contiguous view or a buffer shorter than the call writes.  Each check raises before
the library is called, so these run without a GPU (host tensors throughout; a call's
first device argument is the one refused, the property checks are tested on _dev)."""
import numpy as np
import pytest
import torch

from paper_2206_03015_gb300 import lw


def _det(n_pix=4):
    rng = np.random.Generator(np.random.PCG64(3))
    n = rng.normal(size=(n_pix, 3))
    return lw.Detector(n / np.linalg.norm(n, axis=1, keepdims=True), device="cpu")


def _traj(n_e=2, n_s=10):
    v = lw.lw_traj()
    v.n_e, v.n_s = n_e, n_s
    return lw.Trajectories(torch.empty(0, dtype=torch.uint8), v)


GRID = lw.Grid(0.0, 1e-18, 64)


def test_dev_checks_each_property():
    f64 = torch.zeros(12, dtype=torch.float64)
    with pytest.raises(ValueError, match="float32 given"):
        lw._dev("x", f64.float(), torch.float64)
    with pytest.raises(ValueError, match="contiguous"):
        lw._dev("x", f64.view(6, 2).t(), torch.float64)
    with pytest.raises(ValueError, match="12 elements given, at least 13"):
        lw._dev("x", f64, torch.float64, 13)
    with pytest.raises(ValueError, match="CUDA tensor"):
        lw._dev("x", f64, torch.float64, 12)
    with pytest.raises(ValueError, match="CUDA tensor"):
        lw._dev("x", np.zeros(3))


@pytest.mark.parametrize("precision", [lw.LW_FP64, lw.LW_MIXED, lw.LW_MIXED_KAHAN,
                                       lw.LW_MIXED_F32, lw.LW_MIXED_F32X4])
def test_spectrum_refuses_host_or_mistyped_records(precision):
    det = _det()
    shape, dtype = lw.record_shape(det, GRID, precision)
    rec = torch.zeros(shape, dtype=dtype)
    for call in (lw.lw_spectrum, lw.lw_spectrum_static):
        with pytest.raises(ValueError, match="record: a CUDA tensor"):
            call(rec, precision, det.n_pix, GRID)
        other = torch.float32 if dtype == torch.float64 else torch.float64
        with pytest.raises(ValueError, match="record: .* given, .* required"):
            call(rec.to(other), precision, det.n_pix, GRID)
        with pytest.raises(ValueError, match="record: .* elements given"):
            call(rec.reshape(-1)[:-1], precision, det.n_pix, GRID)


def test_deposit_refuses_host_or_misshapen_records():
    det = _det()
    with pytest.raises(ValueError, match="record: a CUDA tensor"):
        lw.lw_deposit_time_domain(_traj(), det, GRID, lw.LW_FP64)
    shape, dtype = lw.record_shape(det, GRID, lw.LW_MIXED_F32X4)
    with pytest.raises(ValueError, match="record: shape"):
        lw.lw_deposit_time_domain(_traj(), det, GRID, lw.LW_MIXED_F32X4,
                                  record=torch.zeros(shape, dtype=dtype).reshape(-1))


def test_detector_and_outputs_must_be_device_memory():
    det = _det()
    with pytest.raises(ValueError, match="Detector.n_hat: a CUDA tensor"):
        det.c()
    with pytest.raises(ValueError, match="out: a CUDA tensor"):
        lw.lw_grid_bounds(_traj(), det)
    with pytest.raises(ValueError, match="out: a CUDA tensor"):
        lw.lw_spectrum_fdm(_traj(), det, 1e15, 1e13, 8, 1e-17)
    with pytest.raises(ValueError, match="out: 7 elements given"):
        lw.lw_spectrum_fdm(_traj(), det, 1e15, 1e13, 8, 1e-17,
                           out=torch.zeros(7, dtype=torch.float64))


def test_batch_plan_checks_every_record():
    det = _det()
    shape, dtype = lw.record_shape(det, GRID, lw.LW_MIXED)
    with pytest.raises(ValueError, match=r"records\[0\]: a CUDA tensor"):
        lw.lw_batch_plan([_traj()], [det], [GRID], [torch.zeros(shape, dtype=dtype)])


def test_spectrum_grad_checks_its_inputs():
    det = _det()
    nl = GRID.n_bins // 2 + 1
    X = torch.zeros((det.n_pix, 3, nl), dtype=torch.complex128)
    with pytest.raises(ValueError, match="X_save: a CUDA tensor"):
        lw.lw_spectrum_grad(_traj(), det, GRID, X, torch.zeros(det.n_pix, nl))
    with pytest.raises(ValueError, match="X_save: torch.float64 given"):
        lw.lw_spectrum_grad(_traj(), det, GRID, X, torch.zeros(det.n_pix, nl),
                            precision=lw.LW_MIXED)


def test_pusher_checks_state_and_outputs():
    n_e, n_s = 3, 5
    r, u = torch.zeros(n_e, 3, dtype=torch.float64), torch.zeros(n_e, 3, dtype=torch.float64)
    t = torch.zeros(n_s + 1, dtype=torch.float64)
    outs = [torch.zeros(n_e, n_s + 1, 3, dtype=torch.float64) for _ in range(3)]
    laser = (0.8e-6, 0.5, 20e-6, 30e-15)
    with pytest.raises(ValueError, match="r: a CUDA tensor"):
        lw.lw_boris_push(r, u, 0.0, 1e-17, n_s, laser, t, *outs)
    with pytest.raises(ValueError, match="r: torch.float32 given"):
        lw.lw_boris_push(r.float(), u, 0.0, 1e-17, n_s, laser, t, *outs)
    with pytest.raises(ValueError, match="r: 6 elements given, at least 9"):
        lw.lw_boris_push(torch.zeros(n_e, 2, dtype=torch.float64), u, 0.0, 1e-17, n_s, laser,
                         t, *outs)
    with pytest.raises(ValueError, match="r0: a CUDA tensor"):
        lw.lw_boris_push_grad(r, u, 0.0, 1e-17, n_s, laser, *outs)
