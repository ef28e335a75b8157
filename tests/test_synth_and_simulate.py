"""Seeded generators and the simulation readings (ISNR, epsilon, SNR)."""
import math

import numpy as np
import pytest

from oracle import simulate
from paper_1406_0359_gb300 import synth


def test_generators_are_seeded_and_shaped():
    a = synth.sky(64, 1, 3, 10)
    b = synth.sky(64, 1, 3, 10)
    assert np.array_equal(a, b) and a.shape == (64, 64) and a.min() >= 0.0 and a.max() > 0.1
    assert not np.array_equal(a, synth.sky(64, 2, 3, 10))
    uv = synth.uv_coverage(5000, 64, 3)
    assert uv.shape == (5000, 2)
    assert np.array_equal(uv, synth.uv_coverage(5000, 64, 3))
    assert np.all(uv >= -math.pi) and np.all(uv < math.pi)
    assert np.all(np.max(np.abs(uv), axis=1) >= math.pi / 64)  # (0,0) cell suppressed
    # variable density: about 68% of each coordinate within one sigma = pi/4
    frac = np.mean(np.abs(uv[:, 0]) < math.pi / 4)
    assert 0.6 < frac < 0.75


def test_snr_definition():
    x = np.random.default_rng(0).uniform(0, 1, (16, 16))
    assert simulate.snr_db(x, 0.9 * x) == pytest.approx(20.0)
    assert simulate.snr_db(x, 0.99 * x) == pytest.approx(40.0)


def test_input_snr_and_epsilon_rules():
    M = 200_000
    rng = np.random.default_rng(1)
    y0 = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    a, b = synth.noise_draws(M, 7)
    y, sigma = simulate.add_noise(y0, 30.0, a, b)
    n = y - y0
    isnr = 10 * math.log10(np.sum(np.abs(y0) ** 2) / np.sum(np.abs(n) ** 2))
    assert isnr == pytest.approx(30.0, abs=0.05)
    # ||n||^2 ~ sigma^2/2 chi2_2M: eps sits two standard deviations above the mean
    eps = simulate.epsilon(sigma, M)
    z = (eps ** 2 - M * sigma ** 2) / (sigma ** 2 * math.sqrt(M))
    assert z == pytest.approx(2.0, rel=1e-12)
    trials = np.array([np.sum(np.abs(sigma / math.sqrt(2) * (rng.standard_normal(2000) + 1j * rng.standard_normal(2000))) ** 2)
                       for _ in range(4000)])
    e2 = simulate.epsilon(sigma, 2000) ** 2
    assert 0.96 < np.mean(trials <= e2) < 0.99
