"""Simulation protocol and quality metric (oracle, FP64, test infrastructure only).

Section 4 corrupts the visibilities with complex Gaussian noise at a fixed
input SNR (30 dB) and scores reconstructions by SNR, without defining either.
Readings:
* ISNR: sigma = ||Phi x||_2 / sqrt(M) * 10^(-ISNR/20); noise
  n = sigma/sqrt(2) (a + i b) with a, b standard normal;
* epsilon (the l2 bound of problems (2)-(3)): ||n||^2 is sigma^2/2 times a
  chi-square with 2M degrees of freedom, so its mean plus two standard
  deviations gives eps = sigma sqrt(M + 2 sqrt(M));
* SNR(x_hat) = 20 log10(||x|| / ||x - x_hat||).
"""
from __future__ import annotations

import math

import numpy as np


def noise_sigma(y0: np.ndarray, isnr_db: float) -> float:
    return float(np.linalg.norm(y0) / math.sqrt(y0.size) * 10.0 ** (-isnr_db / 20.0))


def add_noise(y0: np.ndarray, isnr_db: float, a: np.ndarray, b: np.ndarray):
    """Return (y, sigma) with y = y0 + sigma/sqrt(2) (a + i b)."""
    sigma = noise_sigma(y0, isnr_db)
    return y0 + sigma / math.sqrt(2.0) * (a + 1j * b), sigma


def epsilon(sigma: float, M: int) -> float:
    return sigma * math.sqrt(M + 2.0 * math.sqrt(M))


def snr_db(x_true: np.ndarray, x_hat: np.ndarray) -> float:
    return 20.0 * math.log10(np.linalg.norm(x_true) / np.linalg.norm(x_true - x_hat))
