"""Python binding of liblw.so (argument marshalling only).

Every function here forwards to the C ABI of ``include/lw.h`` with the same
name; PyTorch supplies device memory and the current CUDA stream.  All
arithmetic of the radiation method runs in the library's CUDA kernels.  There
is no CPU fallback: if the library or a GPU is missing, loading fails with an
error.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass

import torch

from . import build as _build

LW_OK, LW_EINVAL, LW_ESIZE, LW_ECUDA, LW_EUNSUPPORTED, LW_ETIMEOUT = 0, -1, -2, -3, -4, -5
LW_FP64, LW_MIXED, LW_MIXED_KAHAN, LW_MIXED_F32, LW_MIXED_F32X4 = 0, 1, 2, 3, 4
LW_FIELD_ACCEL, LW_FIELD_VELOCITY = 1, 2
LW_ST_BETA, LW_ST_NONFINITE, LW_ST_TIME, LW_ST_CLIP, LW_ST_TA_ORDER, LW_ST_STEP = 1, 2, 4, 8, 16, 32
LW_ST_TIMEOUT, LW_ST_PRECISION = 64, 128
LW_SECTION_FP64, LW_SECTION_MIXED = 1, 2

Q_E = 1.602176634e-19

_ERRORS = {LW_EINVAL: "invalid argument", LW_ESIZE: "workspace too small",
           LW_ECUDA: "CUDA launch failed", LW_EUNSUPPORTED: "unsupported size",
           LW_ETIMEOUT: "device wait timed out"}


class LWError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} returned {code} ({_ERRORS.get(code, 'unknown')})")
        self.code = code


class lw_traj_in(ctypes.Structure):
    _fields_ = [("n_e", ctypes.c_int64), ("n_s", ctypes.c_int64), ("t", ctypes.c_void_p),
                ("t_per_electron", ctypes.c_int32), ("r", ctypes.c_void_p),
                ("beta", ctypes.c_void_p), ("beta_dot", ctypes.c_void_p)]


class lw_traj(ctypes.Structure):
    _fields_ = [("n_e", ctypes.c_int64), ("n_s", ctypes.c_int64),
                ("t_per_electron", ctypes.c_int32), ("sections", ctypes.c_int32),
                ("block", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
                ("t", ctypes.c_void_p), ("r", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("beta_dot", ctypes.c_void_p), ("scan", ctypes.c_void_p),
                ("field", ctypes.c_void_p), ("anchor", ctypes.c_void_p),
                ("ends", ctypes.c_void_p), ("input_status", ctypes.c_void_p),
                ("order", ctypes.c_void_p)]


class lw_batch(ctypes.Structure):
    _fields_ = [("ws", ctypes.c_void_p), ("n_items", ctypes.c_int32), ("n_units", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("field_flags", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("offsets", ctypes.c_int64 * 3)]


class lw_detector(ctypes.Structure):
    _fields_ = [("n_pix", ctypes.c_int64), ("n_hat", ctypes.c_void_p), ("R", ctypes.c_double)]


class lw_grid(ctypes.Structure):
    _fields_ = [("t_min", ctypes.c_double), ("dt_u", ctypes.c_double),
                ("n_bins", ctypes.c_int64)]


class lw_laser(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("a0", ctypes.c_double), ("w0", ctypes.c_double),
                ("fwhm", ctypes.c_double)]


class lw_batch_item(ctypes.Structure):
    _fields_ = [("traj", ctypes.c_void_p), ("det", ctypes.c_void_p), ("grid", lw_grid),
                ("record", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("e_chunk", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None

EXPORTS = ("lw_trajectories_upload", "lw_grid_bounds", "lw_deposit_time_domain", "lw_spectrum",
           "lw_spectrum_grad", "lw_spectrum_static", "lw_batch_plan", "lw_batch_deposit",
           "lw_spectrum_fdm", "lw_boris_push", "lw_boris_push_grad")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblw.so (building it first if needed); raises if unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"liblw.so not built ({path})")
            _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.lw_trajectories_upload.argtypes = [ctypes.POINTER(lw_traj_in), ctypes.c_int32,
                                               ctypes.c_int32, P, ctypes.POINTER(ctypes.c_size_t),
                                               ctypes.POINTER(lw_traj), P]
        lib.lw_grid_bounds.argtypes = [ctypes.POINTER(lw_traj), ctypes.POINTER(lw_detector), P, P]
        lib.lw_deposit_time_domain.argtypes = [ctypes.POINTER(lw_traj), ctypes.POINTER(lw_detector),
                                               ctypes.POINTER(lw_grid), ctypes.c_int32,
                                               ctypes.c_uint32, P, ctypes.c_int32, P, P]
        lib.lw_spectrum.argtypes = [P, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(lw_grid),
                                    ctypes.c_double, P, P, P, ctypes.POINTER(ctypes.c_size_t), P]
        lib.lw_spectrum_grad.argtypes = [ctypes.POINTER(lw_traj), ctypes.POINTER(lw_detector),
                                         ctypes.POINTER(lw_grid), ctypes.c_int32, ctypes.c_uint32,
                                         P, P, ctypes.c_double, P, P, P, P,
                                         ctypes.POINTER(ctypes.c_size_t), P]
        lib.lw_boris_push.argtypes = [P, P, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(lw_laser),
                                      ctypes.c_double, ctypes.c_double, P, P, P, P, P]
        lib.lw_boris_push_grad.argtypes = [P, P, ctypes.c_int64, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int32,
                                           ctypes.POINTER(lw_laser), ctypes.c_double,
                                           ctypes.c_double, P, P, P, P, P, P]
        lib.lw_spectrum_fdm.argtypes = [ctypes.POINTER(lw_traj), ctypes.POINTER(lw_detector),
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                        ctypes.c_double, ctypes.c_double, P, P]
        lib.lw_batch_plan.argtypes = [ctypes.POINTER(lw_batch_item), ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_uint32, P,
                                      ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(lw_batch),
                                      P]
        lib.lw_batch_deposit.argtypes = [ctypes.POINTER(lw_batch), P]
        lib.lw_spectrum_static.argtypes = [P, ctypes.c_int32, ctypes.c_int64,
                                           ctypes.POINTER(lw_grid), ctypes.c_double, P, P, P]
        lib.lw_spectrum_static_capacity.argtypes = []
        lib.lw_spectrum_static_capacity.restype = ctypes.c_size_t
        for f in EXPORTS:
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("paper_2206_03015_gb300 needs a CUDA GPU; no CPU fallback exists")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(fn, rc):
    if rc != LW_OK:
        raise LWError(fn, rc)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _dev(name, t, dtype=None, numel=0):
    """Check a tensor that the library reads or writes as device memory: a contiguous CUDA
    tensor (of ``dtype`` when given) of at least ``numel`` elements.  A host tensor or a
    short buffer would reach a kernel as a bad device address, so it is refused here."""
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: a CUDA tensor is required")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: {t.dtype} given, {dtype} required")
    if not t.is_contiguous():
        raise ValueError(f"{name}: a contiguous tensor is required")
    if t.numel() < numel:
        raise ValueError(f"{name}: {t.numel()} elements given, at least {numel} required")
    if t.device.type != "cuda":
        raise ValueError(f"{name}: a CUDA tensor is required")
    return t


def _ws(name, ws):
    """A caller's workspace: device bytes starting on a 256-byte boundary."""
    _dev(name, ws)
    if ws.data_ptr() % 256:
        raise ValueError(f"{name}: must start on a 256-byte boundary (see workspace())")
    return ws


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """A 256-byte aligned device byte buffer (for the library's workspaces)."""
    return _aligned_bytes(nbytes, device)


def _aligned_bytes(nbytes: int, device) -> torch.Tensor:
    buf = torch.empty(max(int(nbytes), 1) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + max(int(nbytes), 1)]


@dataclass
class Grid:
    """Uniform observer grid t_j = t_min + j dt_u (j = 0..n_bins-1)."""
    t_min: float
    dt_u: float
    n_bins: int

    def c(self) -> lw_grid:
        return lw_grid(float(self.t_min), float(self.dt_u), int(self.n_bins))

    @property
    def omega(self):
        """Angular frequencies omega_l = 2 pi l/(n_bins dt_u), l = 0..n_bins/2."""
        return torch.arange(self.n_bins // 2 + 1, dtype=torch.float64) * (
            2.0 * math.pi / (self.n_bins * self.dt_u))


def grid_from_bounds(t_min: float, t_max: float, n_bins: int) -> Grid:
    """dt_u = (t_max - t_min) / n_bins, so that d_omega = 2 pi / T_u exactly."""
    return Grid(float(t_min), (float(t_max) - float(t_min)) / int(n_bins), int(n_bins))


class Detector:
    """Pixel directions n_hat [n_pix][3] (float64, on the GPU) at radius R."""

    def __init__(self, n_hat, R: float = 1.0, device="cuda"):
        self.n_hat = torch.as_tensor(n_hat, dtype=torch.float64).to(device).contiguous()
        assert self.n_hat.ndim == 2 and self.n_hat.shape[1] == 3
        self.R = float(R)

    @property
    def n_pix(self):
        return self.n_hat.shape[0]

    def c(self) -> lw_detector:
        _dev("Detector.n_hat", self.n_hat, torch.float64, 3 * self.n_pix)
        return lw_detector(self.n_pix, self.n_hat.data_ptr(), self.R)


class Trajectories:
    """Uploaded trajectories: the workspace tensor plus the C view into it."""

    def __init__(self, ws, view: lw_traj):
        self.ws = ws
        self.view = view

    @property
    def n_e(self):
        return self.view.n_e

    @property
    def n_s(self):
        return self.view.n_s

    def mixed_section(self):
        """(scan [n_e, n_s+1, 4] view, field [n_e, n_s+1, 6] copy) float32 of the mixed section
        in the workspace, or None without it.  The field's columns are (beta_x, beta_y,
        beta_dot_x, beta_dot_y, 1 - beta_z, beta_dot_z), stored as a float4 array followed
        by a float2 array."""
        if not self.view.scan:
            return None
        ns1 = self.n_s + 1

        def at(ptr, nbytes):
            off = ptr - self.ws.data_ptr()
            return self.ws[off:off + nbytes].view(torch.float32)
        scan = at(self.view.scan, 16 * self.n_e * ns1).view(self.n_e, ns1, 4)
        f4 = at(self.view.field, 16 * self.n_e * ns1).view(self.n_e, ns1, 4)
        f2 = at(self.view.field + 16 * self.n_e * ns1, 8 * self.n_e * ns1).view(self.n_e, ns1, 2)
        return scan, torch.cat([f4, f2], dim=-1)

    def order(self):
        """The electron visiting order of the deposits (int32 [n_e] view into the
        workspace)."""
        off = self.view.order - self.ws.data_ptr()
        return self.ws[off:off + 4 * self.n_e].view(torch.int32)


def _as_input(x, device):
    if not isinstance(x, torch.Tensor):
        x = torch.from_numpy(x)
    x = x.to(torch.float64)
    if x.device.type == "cpu" and not x.is_pinned():
        x = x.to(device)
    return x.contiguous()


def lw_trajectories_upload(t, r, beta, beta_dot, sections=LW_SECTION_FP64 | LW_SECTION_MIXED,
                           block: int = 512, device="cuda", ws=None) -> Trajectories:
    """Copy trajectories (t, r, beta, beta_dot; CUDA or pinned-CPU float64 tensors,
    or numpy arrays) into the device layout (see lw.h).  ``ws`` may pass a
    previously returned workspace (``Trajectories.ws``) for reuse."""
    _require_cuda()
    lib = load()
    t, r, beta, beta_dot = (_as_input(a, device) for a in (t, r, beta, beta_dot))
    n_e, ns1, three = r.shape
    assert three == 3 and beta.shape == r.shape and beta_dot.shape == r.shape
    t_per_e = 1 if t.ndim == 2 else 0
    inp = lw_traj_in(n_e, ns1 - 1, t.data_ptr(), t_per_e, r.data_ptr(), beta.data_ptr(),
                     beta_dot.data_ptr())
    nbytes = ctypes.c_size_t(0)
    view = lw_traj()
    _check("lw_trajectories_upload",
           lib.lw_trajectories_upload(ctypes.byref(inp), sections, block, None,
                                      ctypes.byref(nbytes), ctypes.byref(view), None))
    if ws is None or ws.numel() < nbytes.value or ws.data_ptr() % 256:
        ws = _aligned_bytes(nbytes.value, device)
    nbytes = ctypes.c_size_t(ws.numel())
    _check("lw_trajectories_upload",
           lib.lw_trajectories_upload(ctypes.byref(inp), sections, block, _ptr(ws),
                                      ctypes.byref(nbytes), ctypes.byref(view), _stream()))
    traj = Trajectories(ws, view)
    traj._inputs = (t, r, beta, beta_dot)   # keep host/pinned sources alive until the copy ran
    return traj


def lw_grid_bounds(traj: Trajectories, det: Detector, out=None):
    """Device double[2] = (t_u^min, t_u^max) of Eqs. (tu_min), (tu_max)."""
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=det.n_hat.device)
    _dev("out", out, torch.float64, 2)
    lib = load()
    d = det.c()
    _check("lw_grid_bounds", lib.lw_grid_bounds(ctypes.byref(traj.view), ctypes.byref(d),
                                                _ptr(out), _stream()))
    return out


def _record_layout(n_pix: int, n_bins: int, precision: int):
    if precision in (LW_FP64, LW_MIXED):
        return (n_pix, 3, n_bins), torch.float64
    if precision == LW_MIXED_F32:
        return (n_pix, 3, n_bins), torch.float32
    if precision == LW_MIXED_F32X4:
        return (n_pix, n_bins, 4), torch.float32
    return (n_pix, 3, n_bins, 2), torch.float32


def _record_arg(name, record, n_pix: int, n_bins: int, precision: int):
    shape, dtype = _record_layout(n_pix, n_bins, precision)
    return _dev(name, record, dtype, math.prod(shape))


def record_shape(det: Detector, grid: Grid, precision: int):
    """(shape, dtype) of the record: FP64 and MIXED accumulate in float64,
    MIXED_KAHAN in (sum, compensation) float32 pairs, MIXED_F32 in float32,
    MIXED_F32X4 in float32 (x, y, z, 0) per pixel and grid point."""
    return _record_layout(det.n_pix, grid.n_bins, precision)


def record_value(record: torch.Tensor, precision: int) -> torch.Tensor:
    """The record as float64 [n_pix][3][n_bins] (sum + compensation for MIXED_KAHAN)."""
    if precision == LW_MIXED_KAHAN:
        return record[..., 0].double() + record[..., 1].double()
    if precision == LW_MIXED_F32X4:
        return record[..., :3].permute(0, 2, 1).double()
    return record.double()


def lw_deposit_time_domain(traj: Trajectories, det: Detector, grid: Grid, precision: int,
                           field_flags: int = LW_FIELD_ACCEL, record=None, accumulate=False,
                           status=None):
    """Algorithm 2 for every pixel; returns the record (see record_shape)."""
    shape, dtype = record_shape(det, grid, precision)
    if record is None:
        record = torch.empty(shape, dtype=dtype, device=det.n_hat.device)
        accumulate = False
    if tuple(record.shape) != shape:
        raise ValueError(f"record: shape {tuple(record.shape)} given, {shape} required")
    _dev("record", record, dtype)
    if status is not None:
        _dev("status", status, torch.int32, 1)
    lib = load()
    d = det.c()
    g = grid.c()
    _check("lw_deposit_time_domain",
           lib.lw_deposit_time_domain(ctypes.byref(traj.view), ctypes.byref(d), ctypes.byref(g),
                                      precision, field_flags, _ptr(record), int(bool(accumulate)),
                                      _ptr(status), _stream()))
    return record


def spectrum_workspace_bytes(precision: int, n_pix: int, grid: Grid) -> int:
    lib = load()
    nbytes = ctypes.c_size_t(0)
    g = grid.c()
    _check("lw_spectrum", lib.lw_spectrum(None, precision, n_pix, ctypes.byref(g), Q_E, None,
                                          None, None, ctypes.byref(nbytes), None))
    return nbytes.value


def lw_spectrum(record, precision: int, n_pix: int, grid: Grid, q: float = Q_E, want_X=False,
                ws=None, out=None):
    """S [n_pix][n_bins/2+1] (FP64 or FP32) and optionally X' [n_pix][3][n_bins/2+1] complex."""
    _record_arg("record", record, n_pix, grid.n_bins, precision)
    dev = record.device
    dtype = torch.float64 if precision == LW_FP64 else torch.float32
    nl = grid.n_bins // 2 + 1
    if out is not None:
        _dev("out", out, dtype, n_pix * nl)
    if ws is not None:
        _ws("ws", ws)
    lib = load()
    S = out if out is not None else torch.empty((n_pix, nl), dtype=dtype, device=dev)
    X = torch.empty((n_pix, 3, nl, 2), dtype=dtype, device=dev) if want_X else None
    need = spectrum_workspace_bytes(precision, n_pix, grid)
    if ws is None or ws.numel() < need:
        ws = _aligned_bytes(need, dev)
    nbytes = ctypes.c_size_t(ws.numel())
    g = grid.c()
    _check("lw_spectrum", lib.lw_spectrum(_ptr(record), precision, n_pix, ctypes.byref(g), q,
                                          _ptr(S), _ptr(X), _ptr(ws), ctypes.byref(nbytes),
                                          _stream()))
    if want_X:
        return S, torch.view_as_complex(X)
    return S


def lw_spectrum_grad(traj: Trajectories, det: Detector, grid: Grid, X_save, dL_dS,
                     q: float = Q_E, out=None, field_flags: int = LW_FIELD_ACCEL,
                     precision: int | None = None):
    """Adjoint of deposit + spectrum.  X_save: [n_pix][3][n_bins/2+1] from
    lw_spectrum(..., want_X=True), complex128 for LW_FP64 or complex64 for a mixed mode;
    precision defaults to LW_FP64 or LW_MIXED after X_save's type.  dL_dS: float64
    [n_pix][n_bins/2+1].  Returns (dL/dr, dL/dbeta, dL/dbeta_dot), each float64
    [n_e][n_s+1][3] (added to ``out`` when given)."""
    dev = det.n_hat.device
    shape = (traj.n_e, traj.n_s + 1, 3)
    if out is None:
        out = tuple(torch.zeros(shape, dtype=torch.float64, device=dev) for _ in range(3))
    X = torch.view_as_real(X_save.contiguous()) if X_save.is_complex() else X_save.contiguous()
    if precision is None:
        precision = LW_FP64 if X.dtype == torch.float64 else LW_MIXED
    nl = grid.n_bins // 2 + 1
    _dev("X_save", X, torch.float64 if precision == LW_FP64 else torch.float32,
         det.n_pix * 3 * nl * 2)
    g = _dev("dL_dS", dL_dS.to(torch.float64).contiguous(), numel=det.n_pix * nl)
    for i, o in enumerate(out):
        _dev(f"out[{i}]", o, torch.float64, math.prod(shape))
    lib = load()
    d = det.c()
    gr = grid.c()
    nbytes = ctypes.c_size_t(0)
    _check("lw_spectrum_grad", lib.lw_spectrum_grad(ctypes.byref(traj.view), ctypes.byref(d),
                                                    ctypes.byref(gr), precision, field_flags, None,
                                                    None, q, None, None, None, None,
                                                    ctypes.byref(nbytes), None))
    ws = _aligned_bytes(nbytes.value, dev)
    _check("lw_spectrum_grad", lib.lw_spectrum_grad(ctypes.byref(traj.view), ctypes.byref(d),
                                                    ctypes.byref(gr), precision, field_flags,
                                                    _ptr(X), _ptr(g), q, _ptr(out[0]),
                                                    _ptr(out[1]), _ptr(out[2]), _ptr(ws),
                                                    ctypes.byref(nbytes), _stream()))
    return out


class BatchPlan:
    """A planned batched deposit (see lw_batch_plan in lw.h); keeps everything the
    device plan points to alive."""

    def __init__(self, ws, plan, keep):
        self.ws = ws
        self.plan = plan
        self._keep = keep


def lw_batch_plan(trajs, dets, grids, records, precision=LW_MIXED, field_flags=LW_FIELD_ACCEL,
                  statuses=None, e_chunks=None) -> BatchPlan:
    """Plan one persistent launch over several variants (lists of equal length)."""
    n = len(trajs)
    for v in range(n):
        _record_arg(f"records[{v}]", records[v], dets[v].n_pix, grids[v].n_bins, precision)
        if statuses is not None:
            _dev(f"statuses[{v}]", statuses[v], torch.int32, 1)
    lib = load()
    items = (lw_batch_item * n)()
    dets_c = [d.c() for d in dets]
    for v in range(n):
        items[v].traj = ctypes.addressof(trajs[v].view)
        items[v].det = ctypes.addressof(dets_c[v])
        items[v].grid = grids[v].c()
        items[v].record = records[v].data_ptr()
        items[v].status = statuses[v].data_ptr() if statuses is not None else None
        items[v].e_chunk = int(e_chunks[v]) if e_chunks is not None else 0
    nbytes = ctypes.c_size_t(0)
    plan = lw_batch()
    _check("lw_batch_plan", lib.lw_batch_plan(items, n, precision, field_flags, None,
                                              ctypes.byref(nbytes), ctypes.byref(plan), None))
    dev = dets[0].n_hat.device
    ws = _aligned_bytes(nbytes.value, dev)
    _check("lw_batch_plan", lib.lw_batch_plan(items, n, precision, field_flags, _ptr(ws),
                                              ctypes.byref(nbytes), ctypes.byref(plan),
                                              _stream()))
    return BatchPlan(ws, plan, (trajs, dets, dets_c, records, statuses))


def lw_batch_deposit(bp: BatchPlan):
    """Zero the records and run the persistent deposit on the current stream."""
    lib = load()
    _check("lw_batch_deposit", lib.lw_batch_deposit(ctypes.byref(bp.plan), _stream()))


def lw_spectrum_fdm(traj: Trajectories, det: Detector, omega0: float, d_omega: float,
                    n_omega: int, dt: float, q: float = Q_E, out=None):
    """Frequency-domain method (Eq. inty_dft) on omega_w = omega0 + w d_omega; float64
    [n_pix][n_omega]."""
    S = out if out is not None else torch.empty((det.n_pix, int(n_omega)), dtype=torch.float64,
                                                device=det.n_hat.device)
    _dev("out", S, torch.float64, det.n_pix * int(n_omega))
    lib = load()
    d = det.c()
    _check("lw_spectrum_fdm", lib.lw_spectrum_fdm(ctypes.byref(traj.view), ctypes.byref(d),
                                                  float(omega0), float(d_omega), int(n_omega),
                                                  float(dt), float(q), _ptr(S), _stream()))
    return S


M_E = 9.1093837015e-31


def lw_boris_push(r, u, t0: float, dt: float, n_steps: int, laser, t_out, r_out, beta_out,
                  bdot_out, charge: float = -Q_E, mass: float = M_E, step0: int = 0):
    """Advance (r, u) [n_e, 3] (float64 CUDA tensors, in place) by n_steps Boris steps in the
    Gaussian laser (lam, a0, w0, fwhm) and write the n_steps+1 samples into the outputs
    (t_out [n_steps+1], r_out/beta_out/bdot_out [n_e, n_steps+1, 3]); sample s is at time
    t0 + dt (step0 + s)."""
    n_e = r.shape[0]
    _dev("r", r, torch.float64, 3 * n_e)
    _dev("u", u, torch.float64, 3 * n_e)
    _dev("t_out", t_out, torch.float64, int(n_steps) + 1)
    for name, o in (("r_out", r_out), ("beta_out", beta_out), ("bdot_out", bdot_out)):
        _dev(name, o, torch.float64, 3 * n_e * (int(n_steps) + 1))
    lib = load()
    L = lw_laser(float(laser[0]), float(laser[1]), float(laser[2]), float(laser[3]))
    _check("lw_boris_push", lib.lw_boris_push(_ptr(r), _ptr(u), r.shape[0], float(t0),
                                              float(dt), int(step0), int(n_steps),
                                              ctypes.byref(L),
                                              float(charge), float(mass), _ptr(t_out),
                                              _ptr(r_out), _ptr(beta_out), _ptr(bdot_out),
                                              _stream()))


def lw_boris_push_grad(r0, u0, t0: float, dt: float, n_steps: int, laser, dL_dr, dL_dbeta,
                       dL_dbeta_dot, charge: float = -Q_E, mass: float = M_E, out=None):
    """Gradient through lw_boris_push from (r0, u0) (float64 CUDA tensors [n_e, 3], read
    only) over n_steps steps: given dL/d(r, beta, beta_dot) [n_e, n_steps+1, 3], returns
    (dL/du0 [n_e, 3], dL/d(a0, w0) [2]) (added to ``out`` when given)."""
    dev = u0.device
    n_e = u0.shape[0]
    if out is None:
        out = (torch.zeros_like(u0, dtype=torch.float64),
               torch.zeros(2, dtype=torch.float64, device=dev))
    _dev("r0", r0.contiguous(), torch.float64, 3 * n_e)
    _dev("u0", u0.contiguous(), torch.float64, 3 * n_e)
    gr, gb, ga = (x.contiguous() for x in (dL_dr, dL_dbeta, dL_dbeta_dot))
    for name, x in (("dL_dr", gr), ("dL_dbeta", gb), ("dL_dbeta_dot", ga)):
        _dev(name, x, torch.float64, 3 * n_e * (int(n_steps) + 1))
    _dev("out[0]", out[0], torch.float64, 3 * n_e)
    _dev("out[1]", out[1], torch.float64, 2)
    lib = load()
    L = lw_laser(float(laser[0]), float(laser[1]), float(laser[2]), float(laser[3]))
    _check("lw_boris_push_grad",
           lib.lw_boris_push_grad(_ptr(r0.contiguous()), _ptr(u0.contiguous()), u0.shape[0],
                                  float(t0), float(dt), int(n_steps), ctypes.byref(L),
                                  float(charge), float(mass), _ptr(gr), _ptr(gb), _ptr(ga),
                                  _ptr(out[0]), _ptr(out[1]), _stream()))
    return out


def lw_spectrum_static(record, precision: int, n_pix: int, grid: Grid, q: float = Q_E,
                       want_X=False, out=None):
    """lw_spectrum without a workspace argument: the library's fixed device scratch
    array is used instead (see include/lw.h); nothing is allocated by the library.
    Output tensors are allocated here unless passed in."""
    _record_arg("record", record, n_pix, grid.n_bins, precision)
    dev = record.device
    dtype = torch.float64 if precision == LW_FP64 else torch.float32
    nl = grid.n_bins // 2 + 1
    if out is not None:
        _dev("out", out, dtype, n_pix * nl)
    lib = load()
    S = out if out is not None else torch.empty((n_pix, nl), dtype=dtype, device=dev)
    X = torch.empty((n_pix, 3, nl, 2), dtype=dtype, device=dev) if want_X else None
    g = grid.c()
    rc = lib.lw_spectrum_static(_ptr(record), precision, n_pix, ctypes.byref(g), q, _ptr(S),
                                _ptr(X), _stream())
    if rc == LW_ESIZE:
        cap = lib.lw_spectrum_static_capacity()
        raise LWError("lw_spectrum_static", rc) from ValueError(
            f"this transform needs more scratch than the fixed {cap} bytes; use lw_spectrum")
    _check("lw_spectrum_static", rc)
    if want_X:
        return S, torch.view_as_complex(X)
    return S

