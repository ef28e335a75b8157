"""The CG operator Re(Phi^H Phi) on the GPU (purify_gram), both forms, against
the oracle's NUFFT and the exact NUDFT normal operator."""
import numpy as np
import pytest
import torch

from oracle.nudft import nudft_matrix
from oracle.nufft import NUFFT
from paper_1406_0359_gb300 import synth
from tests._gpu import TOL, host, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()


def make_op(uv, n, prec):
    from paper_1406_0359_gb300.binding import Operator

    return Operator(torch.as_tensor(uv).cuda(), n, 2, prec)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n,M,seed", [(16, 700, 3), (32, 2500, 4)])
def test_gram_forms_match_exact_normal_operator(prec, n, M, seed):
    uv = synth.uv_coverage(M, n, seed)
    A = nudft_matrix(uv, n)
    x = synth.random_image(n, seed)
    exact = np.real(A.conj().T @ (A @ x.reshape(-1))).reshape(n, n)
    nufft = NUFFT(uv, n).gram_real(x)
    op = make_op(uv, n, prec)
    g0 = host(op.gram(to_dev(x, prec), mode=0))
    g1 = host(op.gram(to_dev(x, prec), mode=1))
    assert rel(g0, nufft) < TOL[prec]
    # the convolution form is the exact normal operator up to the NUFFT error of the PSF
    assert rel(g1, exact) < (1e-5 if prec == "fp32" else 1e-6)
    assert rel(g1, nufft) < (1e-5 if prec == "fp32" else 1e-6)


@pytest.mark.parametrize("n,M,seed", [(64, 4096, 1), (256, 131072, 2)])
def test_gram_convolution_at_config_sizes(n, M, seed):
    uv = synth.uv_coverage(M, n, seed)
    x = synth.sky(n, seed, 3, 10)
    ref = NUFFT(uv, n).gram_real(x)
    op = make_op(uv, n, "fp32")
    assert rel(host(op.gram(to_dev(x, "fp32"), mode=1)), ref) < 1e-5
    assert rel(host(op.gram(to_dev(x, "fp32"), mode=0)), ref) < 1e-5


def test_gram_convolution_symmetric_psd():
    n, M = 64, 3000
    uv = synth.uv_coverage(M, n, 8)
    op = make_op(uv, n, "fp64")
    a, b = synth.random_image(n, 1), synth.random_image(n, 2)
    ga = host(op.gram(to_dev(a, "fp64"), mode=1))
    gb = host(op.gram(to_dev(b, "fp64"), mode=1))
    assert abs(np.sum(b * ga) - np.sum(a * gb)) < 1e-10 * abs(np.sum(a * ga))
    assert np.sum(a * ga) > 0


def test_gram_forms_agree_at_full_size():
    """1024^2 image, 4,194,304 uv points (FP32): the convolution form, whose
    PSF comes from the operator on the 4096^2 grid, agrees with the NUFFT
    form (checked against the oracle at smaller sizes) and stays symmetric."""
    n, M = 1024, 4194304
    uv = synth.uv_coverage(M, n, 3)
    op = make_op(uv, n, "fp32")
    a, b = synth.sky(n, 3, 12, 160), synth.random_image(n, 5)
    g0 = host(op.gram(to_dev(a, "fp32"), mode=0))
    g1 = host(op.gram(to_dev(a, "fp32"), mode=1))
    assert rel(g1, g0) < 1e-5
    gb = host(op.gram(to_dev(b, "fp32"), mode=1))
    assert abs(np.sum(b * g1) - np.sum(a * gb)) < 1e-5 * abs(np.sum(a * g1))


@pytest.mark.parametrize("n,M,seed", [(64, 4096, 1), (128, 20000, 5)])
def test_gram_convolution_matches_cufft(n, M, seed):
    """Cross-check of the library's FFT passes against cuFFT (torch.fft on the
    GPU): the composite operator of Section 3 rebuilt from the oracle's PSF
    k = Re Phi_2n^H(1) on the 2n x 2n image, embedded circulantly on the
    K = 2n grid (offset d at index d mod K), its spectrum's real part (the
    even part of k), and the image placed at pixel index p mod K with p the
    centred pixel coordinate; out = Re F^-1(khat F(x)) cropped back."""
    uv = synth.uv_coverage(M, n, seed)
    x = synth.random_image(n, seed)
    K = 2 * n
    psf = NUFFT(uv, 2 * n).phi_adj_real(np.ones(M))  # offsets d in [-n, n) at index d + n
    emb = np.roll(psf, (-n, -n), axis=(0, 1))  # index d mod K
    dev = torch.device("cuda")
    khat = torch.fft.fft2(torch.as_tensor(emb, dtype=torch.complex128, device=dev)).real
    q = (np.arange(n) - n // 2) % K
    grid = torch.zeros((K, K), dtype=torch.complex128, device=dev)
    grid[np.ix_(q, q)] = torch.as_tensor(x, dtype=torch.complex128, device=dev)
    conv = torch.fft.ifft2(khat * torch.fft.fft2(grid)).real[np.ix_(q, q)]
    ref = conv.cpu().numpy()
    for prec, tol in (("fp32", 1e-5), ("fp64", 1e-10)):
        op = make_op(uv, n, prec)
        assert rel(host(op.gram(to_dev(x, prec), mode=1)), ref) < tol
        op.close()
