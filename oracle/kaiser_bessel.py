"""Kaiser-Bessel interpolation kernel (oracle, FP64, test infrastructure only).

Section 4 computes the measurement operator with an NUFFT (image pixels to
visibilities at off-grid uv points); here its interpolation kernel is
Kaiser-Bessel with support J and 2x oversampling.  The paper does not give beta; the
reading used is the Beatty et al. (2005) rule
    beta = pi * sqrt((J/alpha)^2 (alpha - 1/2)^2 - 0.8),
which is 18.639 for J = 8, alpha = 2.
"""
from __future__ import annotations

import math

import numpy as np


def i0_series(z: np.ndarray) -> np.ndarray:
    """Modified Bessel function I0 from its defining power series
    I0(z) = sum_k (z^2/4)^k / (k!)^2, summed until terms fall below 1e-18 of
    the partial sum (all terms are positive, so there is no cancellation)."""
    z = np.asarray(z, dtype=np.float64)
    q = z * z / 4.0
    term = np.ones_like(q)
    total = np.ones_like(q)
    k = 0
    while True:
        k += 1
        term = term * q / (k * k)
        total = total + term
        if np.all(term <= 1e-18 * total):
            break
        if k > 500:
            raise RuntimeError("I0 series did not converge")
    return total


def beatty_beta(J: int, alpha: float) -> float:
    """Beatty et al. (2005) shape parameter for support J, oversampling alpha."""
    return math.pi * math.sqrt((J / alpha) ** 2 * (alpha - 0.5) ** 2 - 0.8)


def kb(s: np.ndarray, J: int, beta: float) -> np.ndarray:
    """Kernel value at offset s (grid cells): I0(beta sqrt(1-(2s/J)^2)) / I0(beta)
    for |s| <= J/2, zero outside."""
    s = np.asarray(s, dtype=np.float64)
    arg = 1.0 - (2.0 * s / J) ** 2
    inside = arg >= 0.0
    val = i0_series(beta * np.sqrt(np.where(inside, arg, 0.0))) / i0_series(np.array(beta))
    return np.where(inside, val, 0.0)


def kb_hat(xi: np.ndarray, J: int, beta: float) -> np.ndarray:
    """Continuous Fourier transform int kb(s) exp(-2 pi i s xi) ds of the
    normalised kernel, xi in cycles per grid cell:
        J / I0(beta) * sinh(r) / r,  r = sqrt(beta^2 - (pi J xi)^2),
    continued by sin(r')/r' with r' = sqrt((pi J xi)^2 - beta^2) past the
    branch point (the closed form for the Kaiser-Bessel window)."""
    xi = np.asarray(xi, dtype=np.float64)
    d = beta * beta - (math.pi * J * xi) ** 2
    out = np.empty_like(xi)
    pos = d > 1e-12
    neg = d < -1e-12
    mid = ~(pos | neg)
    r = np.sqrt(d[pos])
    out[pos] = np.sinh(r) / r
    r2 = np.sqrt(-d[neg])
    out[neg] = np.sin(r2) / r2
    out[mid] = 1.0
    return out * J / i0_series(np.array(beta))
