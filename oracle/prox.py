"""Closed-form proximity operators (oracle, FP64, test infrastructure only).

Equation (7) defines prox_f(x) = argmin_z f(z) + ||x - z||^2 / 2.  The three
functions of the splitting (6) have closed-form proxes (the paper defers the
derivation to its reference [carrillo13b]; these are the textbook forms):

* f_1 = ||W .||_1 (scaled by gamma): soft thresholding at gamma * w_j;
  at |v| = threshold the result is 0 (reading);
* f_2 = indicator of the positive orthant: componentwise max(v, 0);
* f_3 = indicator of the l2 ball {z : ||z - y|| <= eps}: radial projection,
  v itself when ||v - y|| <= eps.
"""
from __future__ import annotations

import numpy as np


def soft_threshold(v: np.ndarray, tau) -> np.ndarray:
    """prox of tau-weighted l1: sign(v) max(|v| - tau, 0)."""
    return np.sign(v) * np.maximum(np.abs(v) - tau, 0.0)


def proj_positive(v: np.ndarray) -> np.ndarray:
    """Projection onto R_+^N."""
    return np.maximum(v, 0.0)


def proj_l2_ball(v: np.ndarray, y: np.ndarray, eps: float) -> np.ndarray:
    """Projection of v onto {z : ||z - y||_2 <= eps} (real or complex)."""
    d = v - y
    s = float(np.sqrt(np.sum(np.abs(d) ** 2)))
    if s <= eps:
        return np.array(v, copy=True)
    return y + d * (eps / s)
