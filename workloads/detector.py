"""Far-field detector directions.

A pixel direction is parametrised as in the paper's observer sketch,
n = (sin theta_x, cos theta_x sin theta_y, cos theta_x cos theta_y).
"""
from __future__ import annotations

import numpy as np


def n_from_angles(theta_x, theta_y) -> np.ndarray:
    tx = np.asarray(theta_x, dtype=np.float64)
    ty = np.asarray(theta_y, dtype=np.float64)
    return np.stack([np.sin(tx), np.cos(tx) * np.sin(ty), np.cos(tx) * np.cos(ty)], axis=-1)


def detector_grid(nx: int, ny: int, half_x: float, half_y: float | None = None):
    """nx*ny cell-centred pixels over theta_x in [-half_x, half_x], theta_y likewise.

    Returns (n_hat [nx*ny][3] float64, theta_x [nx*ny], theta_y [nx*ny]); pixel
    index = iy*nx + ix.
    """
    if half_y is None:
        half_y = half_x
    tx = (np.arange(nx) + 0.5) / nx * 2.0 * half_x - half_x
    ty = (np.arange(ny) + 0.5) / ny * 2.0 * half_y - half_y
    TX, TY = np.meshgrid(tx, ty, indexing="xy")
    TX = TX.reshape(-1)
    TY = TY.reshape(-1)
    return np.ascontiguousarray(n_from_angles(TX, TY)), TX, TY


def detector_ring(n: int, theta_x: float = 0.0, half_y: float = 1.0):
    """A line of n directions with theta_x fixed and theta_y in [-half_y, half_y]."""
    ty = np.linspace(-half_y, half_y, n)
    return np.ascontiguousarray(n_from_angles(np.full(n, theta_x), ty)), ty
