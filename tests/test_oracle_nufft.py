"""Pins for the oracle's Kaiser-Bessel NUFFT (Section 4 measurement operator)."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

from oracle import kaiser_bessel as kbm
from oracle.nudft import nudft, nudft_adj, nudft_matrix
from oracle.nufft import NUFFT
from paper_1406_0359_gb300 import synth


def test_i0_series_matches_library():
    z = np.linspace(0.0, 30.0, 301)
    ours = kbm.i0_series(z)
    ref = scipy.special.i0(z)
    assert np.max(np.abs(ours / ref - 1.0)) < 1e-14


def test_kb_shape():
    J, beta = 8, kbm.beatty_beta(8, 2.0)
    assert kbm.kb(np.array(0.0), J, beta) == pytest.approx(1.0, abs=0, rel=1e-15)
    edge = kbm.kb(np.array([4.0, -4.0]), J, beta)
    assert np.allclose(edge, 1.0 / scipy.special.i0(beta), rtol=1e-13)
    assert np.all(kbm.kb(np.array([4.0001, -5.0, 100.0]), J, beta) == 0.0)
    s = np.linspace(-4, 4, 81)
    assert np.allclose(kbm.kb(s, J, beta), kbm.kb(-s, J, beta), rtol=0, atol=0)


@pytest.mark.parametrize("xi", [0.0, 0.01, 0.1, 0.25, 0.5, 0.9])
def test_kb_hat_is_the_fourier_transform(xi):
    """Closed-form kernel transform vs numerical quadrature of the kernel."""
    J, beta = 8, kbm.beatty_beta(8, 2.0)
    f = lambda s: float(kbm.kb(np.array(s), J, beta)) * math.cos(2 * math.pi * s * xi)
    ref, _ = scipy.integrate.quad(f, -J / 2, J / 2, epsabs=1e-14, epsrel=1e-13, limit=200)
    ours = float(kbm.kb_hat(np.array([xi]), J, beta)[0])
    assert ours == pytest.approx(ref, rel=1e-9, abs=1e-13)


@pytest.mark.parametrize("n,M", [(8, 300), (16, 800), (32, 2000)])
def test_nufft_matches_exact_nudft(n, M):
    uv = synth.uv_coverage(M, n, 7 + n)
    op = NUFFT(uv, n)
    x = synth.random_image(n, n)
    y = op.phi(x)
    ref = nudft(x, uv)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err < 1e-6, err
    v = synth.random_vis(M, n + 1)
    xa = op.phi_adj(v)
    refa = nudft_adj(v, uv, n)
    erra = np.linalg.norm(xa - refa) / np.linalg.norm(refa)
    assert erra < 1e-6, erra


def test_nufft_uniform_edge_points():
    """Samples exactly on grid nodes and at the corners of [-pi, pi)^2."""
    n = 16
    uv = np.array([[-math.pi, -math.pi], [0.0, math.pi / 2], [-math.pi, 0.5],
                   [math.pi - 1e-12, -math.pi + 1e-12], [math.pi / 16, 0.0]])
    op = NUFFT(uv, n)
    x = synth.random_image(n, 2)
    err = np.linalg.norm(op.phi(x) - nudft(x, uv)) / np.linalg.norm(nudft(x, uv))
    assert err < 1e-6


def test_adjoint_identity():
    n, M = 32, 3000
    uv = synth.uv_coverage(M, n, 3)
    op = NUFFT(uv, n)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = synth.random_vis(M, 5)
    lhs = np.vdot(y, op.phi(x))
    rhs = np.vdot(op.phi_adj(y), x)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12
    xr = synth.random_image(n, 9)
    lr = np.real(np.vdot(y, op.phi(xr)))
    rr = np.sum(xr * op.phi_adj_real(y))
    assert abs(lr - rr) / abs(lr) < 1e-12


def test_dense_matrix_and_adjoint_at_n8():
    n, M = 8, 64
    uv = synth.uv_coverage(M, n, 21)
    op = NUFFT(uv, n)
    eye = np.eye(n * n)
    A = np.stack([op.phi(e.reshape(n, n)) for e in eye], axis=1)
    AH = np.stack([op.phi_adj(e).reshape(-1) for e in np.eye(M)], axis=1)
    assert np.max(np.abs(AH - A.conj().T)) < 1e-12 * np.max(np.abs(A))
    exact = nudft_matrix(uv, n)
    assert np.linalg.norm(A - exact) / np.linalg.norm(exact) < 1e-6


class _Mutant(NUFFT):
    pass


@pytest.mark.parametrize("mutation", ["no_deapod", "wrong_fft_sign", "tap_shift", "swap_uv"])
def test_planted_mistakes_are_caught(mutation, monkeypatch):
    """Each plausible slip in the oracle's Phi breaks the NUDFT pin."""
    n, M = 16, 500
    uv = synth.uv_coverage(M, n, 4)
    if mutation == "swap_uv":
        op = NUFFT(uv[:, ::-1].copy(), n)
    else:
        op = NUFFT(uv, n)
    if mutation == "no_deapod":
        op.S = np.ones_like(op.S)
    elif mutation == "wrong_fft_sign":
        import scipy.fft as sfft

        inv = sfft.ifft2
        monkeypatch.setattr(sfft, "fft2", lambda a, workers=None: inv(a) * a.size)
    elif mutation == "tap_shift":
        uv2 = uv + 2 * math.pi / op.K  # every tap one cell off
        op.G = op._interp_matrix(uv2)
    x = synth.random_image(n, 1)
    ref = nudft(x, uv)
    err = np.linalg.norm(op.phi(x) - ref) / np.linalg.norm(ref)
    assert err > 1e-3
