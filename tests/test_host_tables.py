"""The CUDA path's host-side tables against the oracle (no GPU): the library's
C++ host code is compiled into a small program that prints its Kaiser-Bessel
shape, deapodisation weights, per-tap kernel polynomials and Daubechies
filters; each is compared with the oracle's independent computation."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.daubechies import db_lowpass
from oracle.kaiser_bessel import beatty_beta, kb, kb_hat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    out = tmp_path_factory.mktemp("host_tables") / "host_tables"
    src = [os.path.join(ROOT, "tests", "host_tables_main.cpp"),
           os.path.join(ROOT, "paper_1406_0359_gb300", "csrc", "host_math.cpp")]
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", str(out)] + src, check=True)
    return json.loads(subprocess.run([str(out)], check=True, capture_output=True, text=True).stdout)


def test_kaiser_bessel_shape_and_deapodisation(tables):
    J, beta = 8, beatty_beta(8, 2.0)
    assert abs(tables["beta"] - beta) < 1e-14 * beta
    n, K = 64, 128
    ref = 1.0 / kb_hat((np.arange(n) - n // 2) / K, J, beta)
    got = np.array(tables["deapod_64_128"])
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-12


@pytest.mark.parametrize("deg,tol", [(10, 1e-9), (16, 1e-13)])
def test_kernel_polynomials_follow_the_kernel(tables, deg, tol):
    """Tap a at fraction f in [0, 1): kb(f + J/2 - 1 - a) ~= sum_d c[a][d] x^d,
    x = 2f - 1; checked on a grid that the fit never saw."""
    J, beta = 8, beatty_beta(8, 2.0)
    c = np.array(tables["poly%d" % deg]).reshape(J, deg + 1)
    f = (np.arange(997) + 0.37) / 997.0
    x = 2.0 * f - 1.0
    for a in range(J):
        p = np.polynomial.polynomial.polyval(x, c[a])
        assert np.max(np.abs(p - kb(f + J / 2 - 1 - a, J, beta))) < tol, a


def test_daubechies_filters_match_the_oracle(tables):
    for k in range(1, 9):
        got = np.array(tables["db%d" % k])
        assert got.shape == (2 * k,)
        assert np.max(np.abs(got - db_lowpass(k))) < 1e-12, k
