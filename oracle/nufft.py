"""Measurement operator Phi = G F Z S and its adjoint (oracle, FP64).

Test infrastructure only.  Section 4 of the paper states that the
measurement operator is a non-uniform FFT mapping the discrete image to
continuous visibilities; the factorisation Phi = G F Z S (deapodise, zero-pad
to an alpha-times oversampled grid, 2D FFT, Kaiser-Bessel interpolation) is
the standard one the paper's reference [greengard04] builds on.  Readings of
what the paper leaves open:

* pixel origin, sign and scale follow nudft.py: centred pixels, exp(-i k.p),
  no normalisation;
* grid: K = alpha * n cells per axis; a sample at u (radians per pixel) sits
  at grid coordinate t = u K / (2 pi); its J taps are
  j = floor(t) - J/2 + 1, ..., floor(t) + J/2, wrapped mod K, with weight
  kb(t - j), separable in u and v;
* deapodisation S multiplies pixel p by 1 / (kb_hat(p1/K) kb_hat(p2/K)), the
  analytic kernel transform at the pixel's frequency in cycles per cell;
* Z places pixel p at grid index p mod K; F is the unnormalised forward DFT
  (scipy.fft, run on every host core: the transform is the library's).

The adjoint is the exact conjugate transpose of the same matrices; for a
real image the restricted adjoint is its real part (the problem is posed on
R_+^N, problems (2)-(3)).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft
import scipy.sparse as sp

from .kaiser_bessel import beatty_beta, kb, kb_hat


class NUFFT:
    """Phi and Phi^H for a fixed uv coverage and image side n."""

    def __init__(self, uv: np.ndarray, n: int, oversample: int = 2, J: int = 8):
        uv = np.asarray(uv, dtype=np.float64)
        if uv.ndim != 2 or uv.shape[1] != 2:
            raise ValueError("uv must be (M, 2)")
        self.n, self.J, self.alpha = n, J, oversample
        self.M = uv.shape[0]
        K = oversample * n
        self.K = K
        self.beta = beatty_beta(J, oversample)
        p = np.arange(n) - n // 2
        self.q = p % K  # grid index of each pixel row/column (operator Z)
        khat = kb_hat(p / K, J, self.beta)
        self.S = 1.0 / np.outer(khat, khat)  # deapodisation (operator S)
        self.G = self._interp_matrix(uv)

    def _interp_matrix(self, uv: np.ndarray) -> sp.csr_matrix:
        """Sparse M x K^2 interpolation matrix G (J^2 entries per row)."""
        J, K, M = self.J, self.K, self.M
        t = uv * K / (2.0 * math.pi)
        base = np.floor(t).astype(np.int64) - J // 2 + 1
        a = np.arange(J)
        ju = base[:, 0:1] + a  # (M, J)
        jv = base[:, 1:2] + a
        wu = kb(t[:, 0:1] - ju, J, self.beta)
        wv = kb(t[:, 1:2] - jv, J, self.beta)
        cols = ((ju % K)[:, :, None] * K + (jv % K)[:, None, :]).reshape(-1)
        data = (wu[:, :, None] * wv[:, None, :]).reshape(-1)
        indptr = np.arange(M + 1, dtype=np.int64) * (J * J)
        return sp.csr_matrix((data, cols.astype(np.int64), indptr), shape=(M, K * K))

    # --- forward -----------------------------------------------------------
    def zs(self, x: np.ndarray) -> np.ndarray:
        """Z S x: deapodise and zero-pad to the K x K grid."""
        g = np.zeros((self.K, self.K), dtype=np.complex128)
        g[np.ix_(self.q, self.q)] = self.S * x
        return g

    def phi(self, x: np.ndarray) -> np.ndarray:
        """Phi x = G F Z S x for an n x n image (real or complex)."""
        ghat = sfft.fft2(self.zs(x), workers=-1)
        return self.G @ ghat.reshape(-1)

    # --- adjoint -----------------------------------------------------------
    def phi_adj(self, y: np.ndarray) -> np.ndarray:
        """Phi^H y = S Z^T F^H G^H y as a complex n x n image."""
        ghat = (self.G.T @ np.asarray(y, dtype=np.complex128)).reshape(self.K, self.K)
        g = sfft.ifft2(ghat, workers=-1) * (self.K * self.K)  # unnormalised inverse DFT
        return self.S * g[np.ix_(self.q, self.q)]

    def phi_adj_real(self, y: np.ndarray) -> np.ndarray:
        """Adjoint of Phi restricted to real images: Re(Phi^H y)."""
        return self.phi_adj(y).real

    def gram_real(self, x: np.ndarray) -> np.ndarray:
        """Re(Phi^H Phi x) for a real image x."""
        return self.phi_adj_real(self.phi(x))
