"""Seeded synthetic inputs shaped like the paper's simulations (Section 4).

This module draws random numbers and nothing else: it holds none of the
imaging method's arithmetic (no measurement operator, no wavelets, no
proximal steps).  Both the CUDA path and the FP64 oracle take their inputs
from here, so that the two sides see identical skies, uv coverages and noise
draws.

Workloads (all seeds fixed):

* ``sky``: positive extended emission made of Gaussian blobs plus point
  sources whose fluxes follow a truncated power law (Pareto, index 2).  The
  paper's own ground truth (the 30Dor image, Section 4) is not available, so
  this stands in for it.
* ``uv_coverage``: continuous uv points drawn from a 2D Gaussian
  variable-density profile, denser at low spatial frequencies as in the
  paper's random variable-density sampling (Section 4), kept inside
  [-pi, pi)^2, with the (0, 0) cell of the image's Fourier grid suppressed
  (Section 4 removes the (0, 0) component).
* ``noise_draws``: i.i.d. standard normal pairs (a, b); the caller turns them
  into complex noise of the variance its input-SNR rule fixes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = ["Workload", "WORKLOADS", "sky", "uv_coverage", "noise_draws"]


@dataclass(frozen=True)
class Workload:
    """One named synthetic configuration: image side n, visibility count M,
    wavelet levels, SDMM iteration count and seed."""

    name: str
    n: int
    M: int
    levels: int
    t_max: int
    cg_iters: int
    n_reweight: int
    seed: int
    n_blobs: int
    n_points: int
    isnr_db: float = 30.0
    uv_sigma: float = math.pi / 4


WORKLOADS = {
    # 64x64 sky, 4096 uv points, 3 levels, 200 SDMM iterations.
    "small_64": Workload("small_64", 64, 4096, 3, 200, 10, 3, 1, 3, 10),
    # 256x256 sky, M = 2N = 131072 uv points, 4 levels, 500 iterations.
    "paper_256": Workload("paper_256", 256, 131072, 4, 500, 10, 3, 2, 6, 40),
    # 1024x1024 sky, M = 4,194,304 uv points, 2048^2 oversampled grid.
    "large_1024": Workload("large_1024", 1024, 4194304, 4, 20, 10, 0, 3, 12, 160),
}


def sky(n: int, seed: int, n_blobs: int = 3, n_points: int = 10) -> np.ndarray:
    """Positive n x n float64 sky: Gaussian blobs plus power-law point sources.

    Blob centres are uniform in the central 80% of the field, widths
    sigma ~ U[1.5, max(1.5, n/12)] pixels, peak amplitudes ~ U[0.3, 1].  Point
    fluxes follow a Pareto law of index 2 truncated to [0.1, 1] (inverse-CDF
    draw), at uniformly drawn integer pixels.  Every pixel is >= 0.
    """
    rng = np.random.default_rng(seed)
    img = np.zeros((n, n), dtype=np.float64)
    i0 = np.arange(n, dtype=np.float64)[:, None]
    i1 = np.arange(n, dtype=np.float64)[None, :]
    lo, hi = 0.1 * n, 0.9 * n
    for _ in range(n_blobs):
        c0, c1 = rng.uniform(lo, hi, size=2)
        s = rng.uniform(1.5, max(1.5, n / 12.0))
        amp = rng.uniform(0.3, 1.0)
        img += amp * np.exp(-((i0 - c0) ** 2 + (i1 - c1) ** 2) / (2.0 * s * s))
    # truncated Pareto(alpha=2) on [a, b] by inverse CDF
    a, b, alpha = 0.1, 1.0, 2.0
    uu = rng.uniform(0.0, 1.0, size=n_points)
    flux = a * (1.0 - uu * (1.0 - (a / b) ** alpha)) ** (-1.0 / alpha)
    pos = rng.integers(0, n, size=(n_points, 2))
    for (r, c), f in zip(pos, flux):
        img[r, c] += f
    return img


def uv_coverage(M: int, n: int, seed: int, sigma: float = math.pi / 4) -> np.ndarray:
    """M continuous uv points (radians per pixel) as a float64 (M, 2) array.

    Each coordinate is N(0, sigma^2), redrawn until the point lies in
    [-pi, pi)^2 and outside the DC cell max(|u|, |v|) < pi/n.
    """
    rng = np.random.default_rng(seed)
    out = np.empty((0, 2), dtype=np.float64)
    need = M
    while need > 0:
        cand = rng.normal(0.0, sigma, size=(int(need * 1.3) + 64, 2))
        inside = np.all((cand >= -math.pi) & (cand < math.pi), axis=1)
        not_dc = np.max(np.abs(cand), axis=1) >= math.pi / n
        cand = cand[inside & not_dc]
        out = np.concatenate([out, cand[:need]], axis=0)
        need = M - out.shape[0]
    return out


def noise_draws(M: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Two independent length-M standard normal vectors (real, imaginary)."""
    rng = np.random.default_rng(seed + 1_000_003)
    a = rng.standard_normal(M)
    b = rng.standard_normal(M)
    return a, b


def random_image(n: int, seed: int) -> np.ndarray:
    """Dense n x n float64 test image, entries ~ U[-1, 1] (operator tests)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, n))


def random_vis(M: int, seed: int) -> np.ndarray:
    """Length-M complex128 test vector, real and imaginary parts ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(M) + 1j * rng.standard_normal(M)
