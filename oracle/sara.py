"""SARA dictionary Psi = [Psi_1, ..., Psi_9] and its sub-dictionaries
(oracle, FP64, test infrastructure only).

Section 2.2: q = 9 bases side by side -- the identity (Dirac) and the
orthonormal Daubechies wavelets Db1 to Db8 (D = 9N coefficients).  The paper does not write the
normalisation; Section 3 uses Psi Psi^H = I (the composite operator
sum_i L_i^H L_i = Phi^H Phi + 2I), which holds when every one of the q bases
is scaled by 1/sqrt(q) (reading; 1/3 for SARA).  Coefficients are stored
basis-major: block 0 is the Dirac basis, block b (1..8) the Db_b wavelet
coefficients in Mallat layout.

Section 4 compares the same analysis problem with other dictionaries: BP
(Dirac basis alone), BPDb8 (Db8 alone) and BPSA (all nine bases without
reweighting); `bases` selects any subset (0 = Dirac, K = DbK), kept in
increasing order, with the 1/sqrt(q) scaling for its q bases.
"""
from __future__ import annotations

import numpy as np

from .daubechies import db_highpass, db_lowpass
from .dwt import dwt2, idwt2

ALL_BASES = tuple(range(9))
N_BASES = 9
SCALE = 1.0 / 3.0


def _check(bases) -> tuple:
    b = tuple(sorted(set(int(k) for k in bases)))
    if not b or b[0] < 0 or b[-1] > 8:
        raise ValueError("bases must be a non-empty subset of 0..8")
    return b


def analysis(x: np.ndarray, levels: int, bases=ALL_BASES) -> np.ndarray:
    """Psi^H x: (q, n, n) array [Psi_b^H x for b in bases] / sqrt(q); the
    Dirac block is x, block K the Db_K wavelet transform."""
    bases = _check(bases)
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((len(bases),) + x.shape)
    for s, K in enumerate(bases):
        out[s] = x if K == 0 else dwt2(x, db_lowpass(K), db_highpass(K), levels)
    return out / np.sqrt(len(bases))


def synthesis(c: np.ndarray, levels: int, bases=ALL_BASES) -> np.ndarray:
    """Psi c = sum_b Psi_b c_b / sqrt(q) for c of shape (q, n, n)."""
    bases = _check(bases)
    c = np.asarray(c, dtype=np.float64)
    if c.shape[0] != len(bases):
        raise ValueError("one coefficient block per basis")
    x = np.zeros(c.shape[1:])
    for s, K in enumerate(bases):
        x += c[s] if K == 0 else idwt2(c[s], db_lowpass(K), db_highpass(K), levels)
    return x / np.sqrt(len(bases))
