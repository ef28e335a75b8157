"""Pins for the oracle's Daubechies filters, periodic DWT and SARA dictionary."""
import math

import numpy as np
import pytest

from oracle import dwt, sara
from oracle.daubechies import db_highpass, db_lowpass


def test_db1_is_haar():
    assert np.allclose(db_lowpass(1), [1 / math.sqrt(2)] * 2, atol=1e-15)


def test_db2_closed_form():
    s3 = math.sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * math.sqrt(2.0))
    assert np.allclose(db_lowpass(2), ref, atol=1e-14)


@pytest.mark.parametrize("K", range(1, 9))
def test_filter_conditions(K):
    h, g = db_lowpass(K), db_highpass(K)
    assert h.size == 2 * K
    assert h.sum() == pytest.approx(math.sqrt(2.0), abs=1e-13)
    assert (h * h).sum() == pytest.approx(1.0, abs=1e-13)
    for m in range(1, K):
        assert abs(np.dot(h[: 2 * K - 2 * m], h[2 * m:])) < 1e-13
        assert abs(np.dot(h[: 2 * K - 2 * m], g[2 * m:])) < 1e-13
    k = np.arange(2 * K, dtype=np.float64)
    for p in range(K):  # K vanishing moments of the wavelet
        mom = np.sum(g * k ** p)
        scale = np.sum(np.abs(g) * k ** p)
        assert abs(mom) < 1e-11 * scale
    # K zeros at z = -1 (exact division by (1 + z)^K), and minimum phase:
    # the remaining zeros lie inside the unit circle
    quo = h.copy()
    for _ in range(K):
        quo, rem = np.polydiv(quo, [1.0, 1.0])
        assert np.max(np.abs(rem)) < 1e-12
    if quo.size > 1:
        assert np.all(np.abs(np.roots(quo)) < 1.0)


@pytest.mark.parametrize("K", [1, 2, 5, 8])
@pytest.mark.parametrize("n,levels", [(16, 1), (16, 3), (32, 4)])
def test_dwt_orthonormal(K, n, levels):
    h, g = db_lowpass(K), db_highpass(K)
    rng = np.random.default_rng(K * 100 + n)
    x = rng.standard_normal((n, n))
    c = dwt.dwt2(x, h, g, levels)
    assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    assert np.max(np.abs(dwt.idwt2(c, h, g, levels) - x)) < 1e-12
    d = rng.standard_normal((n, n))
    assert np.max(np.abs(dwt.dwt2(dwt.idwt2(d, h, g, levels), h, g, levels) - d)) < 1e-12
    assert np.sum(c * d) == pytest.approx(np.sum(x * dwt.idwt2(d, h, g, levels)), rel=1e-12)


@pytest.mark.parametrize("K", range(1, 9))
def test_constant_image_lives_in_the_low_band(K):
    n, levels = 32, 2
    c = dwt.dwt2(np.full((n, n), 1.5), db_lowpass(K), db_highpass(K), levels)
    a = n >> levels
    # each level multiplies the low-low band of a constant by 2
    assert np.allclose(c[:a, :a], 1.5 * 2 ** levels, atol=1e-12)
    mask = np.ones_like(c, dtype=bool)
    mask[:a, :a] = False
    assert np.max(np.abs(c[mask])) < 1e-12


@pytest.mark.parametrize("K", [2, 3, 4, 6, 8])
def test_polynomial_rows_have_zero_details(K):
    """Level-1 row details vanish on polynomials of degree < K wherever the
    filter does not wrap around the periodic boundary."""
    n = 64
    i = np.arange(n, dtype=np.float64)
    rowpoly = sum((0.3 * (p + 1)) * ((i - 20.0) / 17.0) ** p for p in range(K))
    x = np.tile(rowpoly, (n, 1))  # varies along axis 1 only
    c = dwt._analysis_1d(x, db_lowpass(K), db_highpass(K), axis=1)
    hi = c[:, n // 2:]
    nowrap = [k for k in range(n // 2) if 2 * k + 2 * K - 1 < n]
    assert np.max(np.abs(hi[:, nowrap])) < 1e-9 * np.max(np.abs(x))


def test_sara_tight_frame():
    """Psi Psi^H = I (Section 3, composite operator), Dirac block = x/3."""
    n, levels = 32, 3
    x = np.random.default_rng(3).standard_normal((n, n))
    c = sara.analysis(x, levels)
    assert c.shape == (9, n, n)
    assert np.allclose(c[0], x / 3.0, atol=0)
    assert np.max(np.abs(sara.synthesis(c, levels) - x)) < 1e-12
    assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    d = np.random.default_rng(4).standard_normal((9, n, n))
    assert np.sum(c * d) == pytest.approx(np.sum(x * sara.synthesis(d, levels)), rel=1e-12)


def test_planted_dwt_mistake_is_caught():
    """A high-pass filter without the alternating sign breaks orthonormality."""
    h = db_lowpass(4)
    g_bad = h[::-1].copy()
    x = np.random.default_rng(0).standard_normal((16, 16))
    c = dwt.dwt2(x, h, g_bad, 1)
    assert abs(np.linalg.norm(c) - np.linalg.norm(x)) > 1e-3


SUBSETS = [(0,), (8,), (0, 8), (1, 2, 5), tuple(range(9))]


@pytest.mark.parametrize("bases", SUBSETS)
def test_sub_dictionary_is_a_tight_frame(bases):
    """Every selection of q bases scaled by 1/sqrt(q) keeps Psi Psi^H = I,
    preserves energy and is the adjoint of its synthesis (Section 4's BP,
    BPDb8 and SA dictionaries)."""
    n, levels = 32, 3
    x = np.random.default_rng(5).standard_normal((n, n))
    c = sara.analysis(x, levels, bases)
    assert c.shape == (len(bases), n, n)
    assert np.max(np.abs(sara.synthesis(c, levels, bases) - x)) < 1e-12
    assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    d = np.random.default_rng(6).standard_normal(c.shape)
    assert np.sum(c * d) == pytest.approx(np.sum(x * sara.synthesis(d, levels, bases)), rel=1e-12)


def test_dirac_dictionary_is_the_identity():
    """BP's dictionary: Psi = I exactly (one basis, scale 1)."""
    x = np.random.default_rng(7).standard_normal((16, 16))
    assert np.array_equal(sara.analysis(x, 2, (0,))[0], x)
    assert np.array_equal(sara.synthesis(x[None], 2, (0,)), x)


def test_single_wavelet_basis_is_orthonormal():
    """BPDb8's dictionary is square and orthonormal: Psi^H Psi = I too."""
    n, levels = 16, 2
    c = np.random.default_rng(8).standard_normal((1, n, n))
    assert np.max(np.abs(sara.analysis(sara.synthesis(c, levels, (8,)), levels, (8,)) - c)) < 1e-12


def test_sub_dictionary_blocks_are_rescaled_sara_blocks():
    """A sub-dictionary's blocks are the SARA blocks of the same bases, rescaled
    from 1/3 to 1/sqrt(q); the order is increasing basis index."""
    n, levels = 32, 3
    x = np.random.default_rng(9).standard_normal((n, n))
    full = sara.analysis(x, levels)
    sub = sara.analysis(x, levels, (8, 0, 3))
    for s, K in enumerate((0, 3, 8)):
        assert np.allclose(sub[s] * np.sqrt(3), full[K] * 3, rtol=0, atol=1e-12)


def test_bad_dictionary_rejected():
    with pytest.raises(ValueError):
        sara.analysis(np.zeros((16, 16)), 2, ())
    with pytest.raises(ValueError):
        sara.analysis(np.zeros((16, 16)), 2, (9,))
