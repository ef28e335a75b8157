"""Daubechies orthonormal filters Db1..Db8 (oracle, FP64, test infrastructure only).

Section 2.2: SARA's dictionary concatenates the Dirac basis with the first
eight orthonormal Daubechies bases.  The paper does not list coefficients;
they follow from Daubechies' construction, restated here:

The low-pass filter H(z) = sum_k h_k z^-k of DbK has K zeros at z = -1 and
|H(e^iw)|^2 = 2 cos^2K(w/2) P(sin^2(w/2)) with
    P(y) = sum_{k=0}^{K-1} binom(K-1+k, k) y^k.
Each root y_r of P gives, through y = (2 - z - 1/z)/4, a reciprocal pair of
z-roots; the minimum-phase factor keeps the one inside the unit circle.  So
    H(z) ~ (1 + z^-1)^K prod_r (1 - z_r z^-1),
scaled so that sum_k h_k = sqrt(2).  The high-pass filter is the quadrature
mirror g_k = (-1)^k h_{2K-1-k}.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


@lru_cache(maxsize=None)
def _db_lowpass(K: int) -> tuple:
    if K < 1:
        raise ValueError("K >= 1")
    # P(y) coefficients, highest degree first for np.roots
    coeffs = [math.comb(K - 1 + k, k) for k in range(K)]
    poly = np.array(coeffs[::-1], dtype=np.float64)
    h = np.array([1.0])
    for _ in range(K):
        h = np.convolve(h, [1.0, 1.0])
    if K > 1:
        for y in np.roots(poly):
            # z^2 - (2 - 4y) z + 1 = 0 ; pick |z| < 1
            b = 2.0 - 4.0 * y
            disc = np.sqrt(b * b - 4.0 + 0j)
            z1 = (b + disc) / 2.0
            z2 = (b - disc) / 2.0
            z = z1 if abs(z1) < 1.0 else z2
            h = np.convolve(h, [1.0, -z])
    h = np.real_if_close(h, tol=1e6)
    h = np.real(h).astype(np.float64)
    h = h * (math.sqrt(2.0) / h.sum())
    return tuple(h.tolist())


def db_lowpass(K: int) -> np.ndarray:
    """DbK analysis low-pass filter h (length 2K), minimum phase, sum sqrt(2)."""
    return np.array(_db_lowpass(K))


def db_highpass(K: int) -> np.ndarray:
    """Quadrature-mirror high-pass g_k = (-1)^k h_{2K-1-k}."""
    h = db_lowpass(K)
    L = h.size
    k = np.arange(L)
    return ((-1.0) ** k) * h[L - 1 - k]
