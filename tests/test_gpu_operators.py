"""GPU parity of Phi, Phi^H and Psi^H, Psi against the FP64 oracle, through the C-ABI."""
import math

import numpy as np
import pytest
import torch

from oracle import sara as osara
from oracle.nufft import NUFFT
from paper_1406_0359_gb300 import synth
from tests._gpu import TOL, host, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu

CASES = [(16, 97, 1), (64, 4096, 1), (256, 131072, 2), (128, 5000, 9)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()


def make_op(uv, n, levels, prec):
    from paper_1406_0359_gb300.binding import Operator

    return Operator(torch.as_tensor(uv).cuda(), n, levels, prec)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n,M,seed", CASES)
def test_phi_and_adjoint_match_oracle(prec, n, M, seed):
    uv = synth.uv_coverage(M, n, seed)
    ref = NUFFT(uv, n)
    op = make_op(uv, n, 2, prec)
    x = synth.random_image(n, seed + 10)
    y = synth.random_vis(M, seed + 20)
    yg = host(op.phi(to_dev(x, prec)))
    assert rel(yg, ref.phi(x)) < TOL[prec]
    xg = host(op.phi_adj(to_dev(y, prec)))
    assert rel(xg, ref.phi_adj_real(y)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_edge_coverages(prec):
    n = 32
    K = 2 * n
    cell = 2 * math.pi / K
    uv = np.array([[-math.pi, -math.pi], [0.0, 0.0], [math.pi - 1e-13, math.pi - 1e-13],
                   [3 * cell, -5 * cell], [0.5 * cell, 0.25 * cell], [-math.pi, 0.3],
                   [7.0, -9.0]])  # last point outside [-pi, pi): wrapped
    wrapped = uv.copy()
    wrapped[-1] = np.mod(uv[-1] + math.pi, 2 * math.pi) - math.pi  # only the out-of-range point
    ref = NUFFT(wrapped, n)
    op = make_op(uv, n, 1, prec)
    x = synth.random_image(n, 3)
    assert rel(host(op.phi(to_dev(x, prec))), ref.phi(x)) < TOL[prec]
    y = synth.random_vis(uv.shape[0], 4)
    assert rel(host(op.phi_adj(to_dev(y, prec))), ref.phi_adj_real(y)) < TOL[prec]
    # every point in one tile; a single point
    uv1 = np.full((300, 2), 0.01) + 1e-3 * np.random.default_rng(0).standard_normal((300, 2))
    ref1 = NUFFT(uv1, n)
    op1 = make_op(uv1, n, 1, prec)
    assert rel(host(op1.phi(to_dev(x, prec))), ref1.phi(x)) < TOL[prec]
    y1 = synth.random_vis(300, 5)
    assert rel(host(op1.phi_adj(to_dev(y1, prec))), ref1.phi_adj_real(y1)) < TOL[prec]
    op2 = make_op(uv1[:1], n, 1, prec)
    assert rel(host(op2.phi(to_dev(x, prec))), NUFFT(uv1[:1], n).phi(x)) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n,levels", [(16, 3), (64, 3), (256, 4), (32, 4)])
def test_sara_matches_oracle(prec, n, levels):
    uv = synth.uv_coverage(64, n, 1)
    op = make_op(uv, n, levels, prec)
    x = synth.random_image(n, n)
    c = host(op.sara_fwd(to_dev(x, prec)))
    cref = osara.analysis(x, levels)
    assert rel(c, cref) < TOL[prec]
    d = np.random.default_rng(n).standard_normal((9, n, n))
    xa = host(op.sara_adj(to_dev(d, prec)))
    assert rel(xa, osara.synthesis(d, levels)) < TOL[prec]
    # tight frame on the GPU
    back = host(op.sara_adj(op.sara_fwd(to_dev(x, prec))))
    assert rel(back, x) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_adjoint_identity_on_gpu(prec):
    n, M = 256, 131072
    uv = synth.uv_coverage(M, n, 2)
    op = make_op(uv, n, 4, prec)
    x = synth.random_image(n, 1)
    y = synth.random_vis(M, 2)
    lhs = float(np.real(np.vdot(y, host(op.phi(to_dev(x, prec))))))
    rhs = float(np.sum(x * host(op.phi_adj(to_dev(y, prec)))))
    assert abs(lhs - rhs) / abs(lhs) < (1e-5 if prec == "fp32" else 1e-12)


def test_full_size_phi_sampled_and_adjoint_identity():
    """1024^2 image, 4,194,304 uv points, 2048^2 grid, FP32 (the bench
    configuration): sampled visibilities against the oracle computed one by
    one, and the adjoint identity over all of them."""
    n, M = 1024, 4194304
    uv = synth.uv_coverage(M, n, 3)
    op = make_op(uv, n, 4, "fp32")
    x = synth.sky(n, 3, 12, 160)
    yg = host(op.phi(to_dev(x, "fp32")))
    idx = np.random.default_rng(0).choice(M, 2000, replace=False)
    ref = NUFFT(uv[idx], n).phi(x)
    assert rel(yg[idx], ref) < TOL["fp32"]
    y = synth.random_vis(M, 4)
    xg = host(op.phi_adj(to_dev(y, "fp32")))
    lhs = float(np.real(np.vdot(y, yg)))
    rhs = float(np.sum(x * xg))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_largest_grid_phi_sampled_and_adjoint_identity():
    """2048^2 image on the 4096^2 grid (the largest transform size): sampled
    visibilities against the oracle and the adjoint identity."""
    n, M = 2048, 65536
    uv = synth.uv_coverage(M, n, 6)
    op = make_op(uv, n, 2, "fp32")
    x = synth.sky(n, 6, 12, 320)
    yg = host(op.phi(to_dev(x, "fp32")))
    idx = np.random.default_rng(1).choice(M, 500, replace=False)
    assert rel(yg[idx], NUFFT(uv[idx], n).phi(x)) < TOL["fp32"]
    y = synth.random_vis(M, 7)
    xg = host(op.phi_adj(to_dev(y, "fp32")))
    lhs = float(np.real(np.vdot(y, yg)))
    rhs = float(np.sum(x * xg))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


@pytest.mark.parametrize("prec,tile,chunk", [("fp32", 8, 256), ("fp32", 16, 2048), ("fp64", 8, 512)])
def test_tile_options_keep_parity(prec, tile, chunk):
    from paper_1406_0359_gb300.binding import Operator

    n, M = 64, 4096
    uv = synth.uv_coverage(M, n, 1)
    ref = NUFFT(uv, n)
    op = Operator(torch.as_tensor(uv).cuda(), n, 2, prec, tile=tile, chunk=chunk)
    assert op.info()["tile"] == tile
    x = synth.random_image(n, 3)
    y = synth.random_vis(M, 4)
    assert rel(host(op.phi(to_dev(x, prec))), ref.phi(x)) < TOL[prec]
    assert rel(host(op.phi_adj(to_dev(y, prec))), ref.phi_adj_real(y)) < TOL[prec]


def test_autotuner_returns_a_valid_choice():
    from paper_1406_0359_gb300.binding import purify_autotune

    n, M = 128, 20000
    uv = torch.as_tensor(synth.uv_coverage(M, n, 2)).cuda()
    tile, chunk, ms = purify_autotune(uv, n, 3)
    assert tile in (8, 16) and chunk in (256, 512, 1024, 2048) and ms > 0


def test_repeated_creation_reuses_set_up_memory_deterministically():
    """Operators built one after another (their binning scratch and PSF set-up
    buffers come from the library's set-up pool, reused between creations)
    give the same Phi bit for bit (a gather) and the same Phi^H and
    convolution-form Phi^H Phi up to the order of the gridding's global
    atomic adds."""
    n, M = 128, 20000
    uv = synth.uv_coverage(M, n, 11)
    x = to_dev(synth.sky(n, 11, 3, 10), "fp32")
    y = to_dev(synth.random_vis(M, 12), "fp32")
    outs = []
    for _ in range(3):
        op = make_op(uv, n, 3, "fp32")
        outs.append((host(op.phi(x)), host(op.phi_adj(y)), host(op.gram(x, mode=1))))
        op.close()
    for later in outs[1:]:
        assert np.array_equal(outs[0][0], later[0])
        assert rel(later[1], outs[0][1]) < 1e-6
        assert rel(later[2], outs[0][2]) < 1e-6
