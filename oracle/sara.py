"""SARA dictionary Psi = [Psi_1, ..., Psi_9] (oracle, FP64, test infrastructure only).

Section 2.2: the dictionary concatenates the Dirac basis and the first eight
orthonormal Daubechies bases (q = 9, D = 9N).  The paper does not write the
normalisation; Section 3 uses Psi Psi^H = I (the composite operator
sum_i L_i^H L_i = Phi^H Phi + 2I), which holds when every basis is scaled by
1/sqrt(9) = 1/3 (reading).  Coefficients are stored basis-major: block 0 is
the Dirac basis, block b (1..8) the Db_b wavelet coefficients in Mallat layout.
"""
from __future__ import annotations

import numpy as np

from .daubechies import db_highpass, db_lowpass
from .dwt import dwt2, idwt2

N_BASES = 9
SCALE = 1.0 / 3.0


def analysis(x: np.ndarray, levels: int) -> np.ndarray:
    """Psi^H x: (9, n, n) array [x, W_1 x, ..., W_8 x] / 3."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((N_BASES,) + x.shape)
    out[0] = x
    for K in range(1, 9):
        out[K] = dwt2(x, db_lowpass(K), db_highpass(K), levels)
    return out * SCALE


def synthesis(c: np.ndarray, levels: int) -> np.ndarray:
    """Psi c = (c_0 + sum_b W_b^T c_b) / 3 for c of shape (9, n, n)."""
    c = np.asarray(c, dtype=np.float64)
    x = np.array(c[0], copy=True)
    for K in range(1, 9):
        x += idwt2(c[K], db_lowpass(K), db_highpass(K), levels)
    return x * SCALE
