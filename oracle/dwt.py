"""Periodic orthonormal 2D wavelet transform (oracle, FP64, test infrastructure only).

Each SARA basis Psi_b (b = 1..8) is an L-level periodic DbK wavelet basis
(Section 2.2).  Conventions, which the paper leaves open (readings):

* one analysis step on a length-Lx periodic signal, Lx even:
      lo[k] = sum_m h[m] x[(2k + m) mod Lx],  hi[k] = sum_m g[m] x[(2k + m) mod Lx],
  stored as [lo | hi] (Mallat layout);
* in 2D a level transforms every row (along axis 1), then every column
  (along axis 0), of the current low-low band, which sits in the top-left
  corner; the next level recurses on that corner;
* synthesis is the exact adjoint of analysis, which for these orthonormal
  filters is also its inverse.
"""
from __future__ import annotations

import numpy as np


def _analysis_1d(x: np.ndarray, h: np.ndarray, g: np.ndarray, axis: int) -> np.ndarray:
    """One periodic analysis step along `axis` (direct circular convolution)."""
    x = np.moveaxis(x, axis, -1)
    Lx = x.shape[-1]
    if Lx % 2:
        raise ValueError("length must be even")
    k = np.arange(Lx // 2)
    lo = np.zeros(x.shape[:-1] + (Lx // 2,))
    hi = np.zeros_like(lo)
    for m in range(h.size):
        idx = (2 * k + m) % Lx
        lo += h[m] * x[..., idx]
        hi += g[m] * x[..., idx]
    return np.moveaxis(np.concatenate([lo, hi], axis=-1), -1, axis)


def _synthesis_1d(c: np.ndarray, h: np.ndarray, g: np.ndarray, axis: int) -> np.ndarray:
    """Adjoint of _analysis_1d: scatter each coefficient back through its taps."""
    c = np.moveaxis(c, axis, -1)
    Lx = c.shape[-1]
    lo, hi = c[..., : Lx // 2], c[..., Lx // 2 :]
    k = np.arange(Lx // 2)
    x = np.zeros(c.shape)
    for m in range(h.size):
        idx = (2 * k + m) % Lx
        contrib = h[m] * lo + g[m] * hi
        # idx is a permutation of even or odd positions for each m: no repeats
        x[..., idx] += contrib
    return np.moveaxis(x, -1, axis)


def dwt2(x: np.ndarray, h: np.ndarray, g: np.ndarray, levels: int) -> np.ndarray:
    """L-level periodic 2D analysis, Mallat layout, same shape as x."""
    c = np.array(x, dtype=np.float64, copy=True)
    n0, n1 = c.shape
    for lev in range(levels):
        a0, a1 = n0 >> lev, n1 >> lev
        if a0 % 2 or a1 % 2:
            raise ValueError("image side must be divisible by 2**levels")
        band = c[:a0, :a1]
        band = _analysis_1d(band, h, g, axis=1)
        band = _analysis_1d(band, h, g, axis=0)
        c[:a0, :a1] = band
    return c


def idwt2(c: np.ndarray, h: np.ndarray, g: np.ndarray, levels: int) -> np.ndarray:
    """Adjoint (= inverse) of dwt2."""
    x = np.array(c, dtype=np.float64, copy=True)
    n0, n1 = x.shape
    for lev in reversed(range(levels)):
        a0, a1 = n0 >> lev, n1 >> lev
        band = x[:a0, :a1]
        band = _synthesis_1d(band, h, g, axis=0)
        band = _synthesis_1d(band, h, g, axis=1)
        x[:a0, :a1] = band
    return x
