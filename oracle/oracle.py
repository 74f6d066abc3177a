"""ctypes wrapper around ``oracle.c`` (plain FP64 CPU oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays are numpy
float64, C-contiguous, laid out as documented in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

FLAG_ACCEL = 1
FLAG_VELOCITY = 2
FLAG_EXACT = 4

ST_BETA = 1
ST_NONFINITE = 2
ST_TIME = 4
ST_CLIP = 8
ST_TA_ORDER = 16

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, OpenMP,
    no FMA contraction, no machine-specific flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    D = ctypes.c_double
    lib.oracle_grid_bounds.argtypes = [I64, I64, P, I, P, P, P, I64, P, D, I, P, P]
    lib.oracle_advanced_times.argtypes = [I64, I64, P, I, P, I64, P, D, I, P]
    lib.oracle_fields.argtypes = [I64, I64, P, P, P, I64, P, D, I, P]
    lib.oracle_tdm_deposit.argtypes = [I64, I64, P, I, P, P, P, I64, P, D, D, D, I64,
                                       I, I, P, P]
    lib.oracle_fft.argtypes = [I64, P, P]
    lib.oracle_dft.argtypes = [I64, P, P, P, P]
    lib.oracle_spectrum.argtypes = [I64, I64, P, D, D, P, P]
    lib.oracle_fdm.argtypes = [I64, I64, P, I, P, P, P, I64, P, I64, P, D, D, P]
    lib.oracle_tdm_grad.argtypes = [I64, I64, P, I, P, P, P, I64, P, D, D, I64, P, D, P, P, P]
    for f in ("oracle_grid_bounds", "oracle_advanced_times", "oracle_fields",
              "oracle_tdm_deposit", "oracle_fft", "oracle_dft", "oracle_spectrum",
              "oracle_fdm", "oracle_tdm_grad", "oracle_num_threads"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


def load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


def build_variant(src_text: str, out_path: str) -> None:
    """Compile a modified copy of the oracle source (used by the tests that
    plant mistakes in the oracle to show that the pins catch them)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared",
                    "-fPIC", "-o", out_path, src, "-lm"], check=True)


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


class use_library:
    """Context manager: route every oracle call through another build."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        load()
        self.saved = _lib
        _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class _Traj:
    """Normalised view of a trajectory set (t, r, beta, beta_dot)."""

    def __init__(self, t, r, beta, beta_dot):
        self.r = _f64(r)
        self.beta = _f64(beta) if beta is not None else np.zeros_like(self.r)
        self.beta_dot = _f64(beta_dot) if beta_dot is not None else np.zeros_like(self.r)
        assert self.r.ndim == 3 and self.r.shape[2] == 3
        self.n_e, ns1, _ = self.r.shape
        self.n_s = ns1 - 1
        self.t = _f64(t)
        if self.t.ndim == 1:
            assert self.t.shape[0] == ns1
            self.t_per_e = 0
        else:
            assert self.t.shape == (self.n_e, ns1)
            self.t_per_e = 1


def grid_bounds(t, r, n_hat, R=1.0, flags=FLAG_ACCEL):
    """Eqs. (tu_min), (tu_max): (t_u^min, t_u^max) over all electrons/pixels."""
    lib = load()
    tr = _Traj(t, r, None, None)
    n_hat = _f64(n_hat).reshape(-1, 3)
    lo = ctypes.c_double()
    hi = ctypes.c_double()
    lib.oracle_grid_bounds(tr.n_e, tr.n_s, _ptr(tr.t), tr.t_per_e, _ptr(tr.r), None, None,
                           n_hat.shape[0], _ptr(n_hat), R, flags, ctypes.byref(lo),
                           ctypes.byref(hi))
    return lo.value, hi.value


def advanced_times(t, r, n_hat, R=1.0, flags=FLAG_ACCEL):
    """t_a[m][k][i], Eq. (far_adv) (or Eq. advanced_condition with FLAG_EXACT)."""
    lib = load()
    tr = _Traj(t, r, None, None)
    n_hat = _f64(n_hat).reshape(-1, 3)
    out = np.empty((n_hat.shape[0], tr.n_e, tr.n_s + 1))
    lib.oracle_advanced_times(tr.n_e, tr.n_s, _ptr(tr.t), tr.t_per_e, _ptr(tr.r),
                              n_hat.shape[0], _ptr(n_hat), R, flags, _ptr(out))
    return out


def fields(r, beta, beta_dot, n_hat, R=1.0, flags=FLAG_ACCEL):
    """F[m][k][i][3], Eq. (far_efield) with the constant q/(4 pi eps0 c0 R) removed."""
    lib = load()
    tr = _Traj(np.zeros(np.shape(r)[1]), r, beta, beta_dot)
    n_hat = _f64(n_hat).reshape(-1, 3)
    out = np.empty((n_hat.shape[0], tr.n_e, tr.n_s + 1, 3))
    st = lib.oracle_fields(tr.n_e, tr.n_s, _ptr(tr.r), _ptr(tr.beta), _ptr(tr.beta_dot),
                           n_hat.shape[0], _ptr(n_hat), R, flags, _ptr(out))
    return out, st


def tdm_deposit(t, r, beta, beta_dot, n_hat, t_min, dt_u, n_bins, R=1.0, flags=FLAG_ACCEL,
                rec=None):
    """Algorithm 2 for every pixel.  Returns (rec[n_pix][3][n_bins], status)."""
    lib = load()
    tr = _Traj(t, r, beta, beta_dot)
    n_hat = _f64(n_hat).reshape(-1, 3)
    n_pix = n_hat.shape[0]
    acc = 1
    if rec is None:
        rec = np.zeros((n_pix, 3, int(n_bins)))
        acc = 0
    assert rec.dtype == np.float64 and rec.flags.c_contiguous
    st = ctypes.c_int(0)
    lib.oracle_tdm_deposit(tr.n_e, tr.n_s, _ptr(tr.t), tr.t_per_e, _ptr(tr.r), _ptr(tr.beta),
                           _ptr(tr.beta_dot), n_pix, _ptr(n_hat), R, float(t_min), float(dt_u),
                           int(n_bins), flags, acc, _ptr(rec), ctypes.byref(st))
    return rec, st.value


def fft(x):
    """Radix-2 FFT, X_l = sum_j x_j exp(+2 pi i j l / n)."""
    lib = load()
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real.copy())
    im = np.ascontiguousarray(x.imag.copy())
    rc = lib.oracle_fft(re.shape[0], _ptr(re), _ptr(im))
    if rc != 0:
        raise ValueError("length must be a power of two")
    return re + 1j * im


def dft(x):
    """Direct O(n^2) DFT with the same sign convention."""
    lib = load()
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real.copy())
    im = np.ascontiguousarray(x.imag.copy())
    ore = np.empty_like(re)
    oim = np.empty_like(im)
    lib.oracle_dft(re.shape[0], _ptr(re), _ptr(im), _ptr(ore), _ptr(oim))
    return ore + 1j * oim


Q_E = 1.602176634e-19


def spectrum(rec, dt_u, q=Q_E, want_X=False):
    """S[m][l] = q^2 dt_u^2/(16 pi^3 eps0 c0) sum_c |X_{m,c}(l)|^2, l = 0..N/2."""
    lib = load()
    rec = _f64(rec)
    n_pix, three, n_bins = rec.shape
    assert three == 3
    nl = n_bins // 2 + 1
    S = np.empty((n_pix, nl))
    X = np.empty((n_pix, 3, nl, 2)) if want_X else None
    rc = lib.oracle_spectrum(n_pix, n_bins, _ptr(rec), float(dt_u), float(q), _ptr(S), _ptr(X))
    if rc != 0:
        raise ValueError("n_bins must be a power of two >= 2")
    if want_X:
        return S, X[..., 0] + 1j * X[..., 1]
    return S


def fdm(t, r, beta, beta_dot, n_hat, omega, dt, q=Q_E):
    """Eq. (inty_dft): frequency-domain method, S[m][w]."""
    lib = load()
    tr = _Traj(t, r, beta, beta_dot)
    n_hat = _f64(n_hat).reshape(-1, 3)
    omega = _f64(omega).reshape(-1)
    S = np.empty((n_hat.shape[0], omega.shape[0]))
    st = lib.oracle_fdm(tr.n_e, tr.n_s, _ptr(tr.t), tr.t_per_e, _ptr(tr.r), _ptr(tr.beta),
                        _ptr(tr.beta_dot), n_hat.shape[0], _ptr(n_hat), omega.shape[0],
                        _ptr(omega), float(dt), float(q), _ptr(S))
    return S, st


def tdm_grad(t, r, beta, beta_dot, n_hat, t_min, dt_u, n_bins, g, q=Q_E):
    """Gradient of L = sum g[m][l] S[m][l] (acceleration far field, l = 0..n_bins/2) with
    respect to every sample's r, beta, beta_dot: (dr, dbeta, dbdot) [n_e][n_s+1][3]."""
    lib = load()
    tr = _Traj(t, r, beta, beta_dot)
    n_hat = _f64(n_hat).reshape(-1, 3)
    g = _f64(g).reshape(n_hat.shape[0], int(n_bins) // 2 + 1)
    out = [np.zeros((tr.n_e, tr.n_s + 1, 3)) for _ in range(3)]
    lib.oracle_tdm_grad(tr.n_e, tr.n_s, _ptr(tr.t), tr.t_per_e, _ptr(tr.r), _ptr(tr.beta),
                        _ptr(tr.beta_dot), n_hat.shape[0], _ptr(n_hat), float(t_min),
                        float(dt_u), int(n_bins), _ptr(g), float(q), _ptr(out[0]), _ptr(out[1]),
                        _ptr(out[2]))
    return tuple(out)


def num_threads() -> int:
    return int(load().oracle_num_threads())
