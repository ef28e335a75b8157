"""Conjugate gradient for the SDMM global update (oracle, FP64, test infrastructure only).

Algorithm 1, step 5 solves (sum_i L_i^H L_i) x = sum_i x_i, and the paper
states that it uses a conjugate gradient algorithm (Section 3).  The
iteration count, tolerance and start are not given; reading: a fixed number
of plain Hestenes-Stiefel steps, warm-started from the previous estimate,
with no early exit.  A step whose denominators vanish leaves the iterate
unchanged (alpha = 0 when <p, Ap> = 0, beta = 0 when <r, r> = 0).
"""
from __future__ import annotations

import numpy as np


def cg(apply_A, b: np.ndarray, x0: np.ndarray, iters: int) -> np.ndarray:
    """`iters` CG steps on A x = b (A symmetric positive definite) from x0."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_A(x)
    p = r.copy()
    rr = float(np.vdot(r, r).real)
    for _ in range(iters):
        Ap = apply_A(p)
        pAp = float(np.vdot(p, Ap).real)
        alpha = rr / pAp if pAp > 0.0 else 0.0
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(np.vdot(r, r).real)
        beta = rr_new / rr if rr > 0.0 else 0.0
        p = r + beta * p
        rr = rr_new
    return x
