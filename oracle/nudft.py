"""Exact non-uniform DFT (oracle pin only, FP64, test infrastructure only).

Section 2.1: under the narrow-band, small-field assumptions the visibilities
are Fourier measurements, so the measurement operator is a Fourier matrix
sampled at M continuous spatial frequencies.  Reading of the sign, origin
and normalisation (the paper is silent): pixel (i1, i2) of an n x n image
sits at p = (i1 - n/2, i2 - n/2), and
    y_m = sum_p x_p exp(-i (u_m p1 + v_m p2)),
unnormalised.  The NUFFT in nufft.py approximates exactly this matrix.
"""
from __future__ import annotations

import numpy as np


def nudft_matrix(uv: np.ndarray, n: int) -> np.ndarray:
    """Dense M x n^2 matrix A[m, i1*n + i2] = exp(-i(u_m p1 + v_m p2))."""
    uv = np.asarray(uv, dtype=np.float64)
    p = np.arange(n, dtype=np.float64) - n // 2
    p1 = np.repeat(p, n)
    p2 = np.tile(p, n)
    phase = np.outer(uv[:, 0], p1) + np.outer(uv[:, 1], p2)
    return np.exp(-1j * phase)


def nudft(x: np.ndarray, uv: np.ndarray) -> np.ndarray:
    """Forward exact transform of an n x n image."""
    n = x.shape[0]
    return nudft_matrix(uv, n) @ np.asarray(x).reshape(-1)


def nudft_adj(y: np.ndarray, uv: np.ndarray, n: int) -> np.ndarray:
    """Conjugate transpose of the exact transform, as an n x n complex image."""
    return (nudft_matrix(uv, n).conj().T @ y).reshape(n, n)
