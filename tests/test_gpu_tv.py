"""TV and RWTV (Section 4) on the GPU against the FP64 oracle: fixed-count
SDMM solves with the TV block (64^2 sky, 4096 uv points), the default gamma
rule, and a checkpoint round trip that carries the TV dual."""
import math

import numpy as np
import pytest
import torch

from oracle import sdmm as osdmm
from oracle import simulate
from oracle import tv as otv
from tests._gpu import host, measured_problem, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu

IMG_TOL = {"fp32": 1e-3, "fp64": 1e-9}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()


@pytest.fixture(scope="module")
def small():
    P = measured_problem(64, 4096, 1)
    nu = 1.0 / math.sqrt(osdmm.operator_norm_sq(P["op"], 30))
    P.update(nu=nu, gamma=otv.tv_default_gamma(P["op"], P["y"], nu))
    return P


def make_op(P, prec, tv_iters=20):
    from paper_1406_0359_gb300.binding import Operator

    op = Operator(torch.as_tensor(P["uv"]).cuda(), P["n"], 3, prec)
    op.set_prior("tv", tv_iters)
    return op


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_default_gamma_matches_oracle(small, prec):
    op = make_op(small, prec)
    res = op.solve(to_dev(small["y"], prec), small["eps"], t_max=1, cg_iters=1, nu=small["nu"], gram=0)
    assert res.stats["gamma"] == pytest.approx(small["gamma"], rel=1e-5 if prec == "fp32" else 1e-10)
    op.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("n_rw,tv_iters", [(0, 20), (1, 15)])
def test_tv_and_rwtv_solves_match_oracle(small, prec, n_rw, tv_iters):
    T, cg_iters = 30, 10
    x_ref, rounds = otv.tv_solve(small["op"], small["y"], small["eps"], small["gamma"], T, cg_iters, small["nu"],
                                 tv_iters, n_rw)
    op = make_op(small, prec, tv_iters)
    res = op.solve(to_dev(small["y"], prec), small["eps"], t_max=T, cg_iters=cg_iters, n_reweight=n_rw,
                   gamma=small["gamma"], nu=small["nu"], gram=0)
    xg = host(res.x)
    assert res.stats["iterations"] == T * (n_rw + 1)
    assert rel(xg, x_ref) < IMG_TOL[prec]
    assert abs(simulate.snr_db(small["x_true"], xg) - simulate.snr_db(small["x_true"], x_ref)) < 0.05
    last = rounds[-1].history[-1]
    assert res.stats["objective"] == pytest.approx(last["objective"], rel=10 * IMG_TOL[prec])
    op.close()


def test_tv_with_the_composite_operator_by_convolution(small):
    """gram = 1 (PSF convolution in the CG) against the oracle's NUFFT form:
    they differ by the NUFFT error of the PSF, well inside 1e-3."""
    x_ref, _ = otv.tv_solve(small["op"], small["y"], small["eps"], small["gamma"], 30, 10, small["nu"], 20, 0)
    op = make_op(small, "fp32")
    res = op.solve(to_dev(small["y"], "fp32"), small["eps"], t_max=30, cg_iters=10, gamma=small["gamma"],
                   nu=small["nu"], gram=1)
    assert rel(host(res.x), x_ref) < 1e-3
    op.close()


def test_tv_checkpoint_carries_the_dual(small):
    kw = dict(t_max=20, cg_iters=8, n_reweight=1, gamma=small["gamma"], nu=small["nu"], gram=0)
    y = to_dev(small["y"], "fp64")
    op = make_op(small, "fp64", 7)  # an odd count: the dual leaves the second buffer
    ref = op.solve(y, small["eps"], **kw)
    op.close()
    a = make_op(small, "fp64", 7)
    a.solve_begin(y, small["eps"], **kw)
    a.solve_step(11)
    state = a.save_state()
    a.close()
    b = make_op(small, "fp64", 7)
    b.solve_begin(y, small["eps"], **kw)
    b.load_state(state)
    while not b.solve_step(10):
        pass
    res = b.solve_end()
    b.close()
    assert rel(host(res.x), host(ref.x)) < 1e-11


def test_prior_argument_checks(small):
    from paper_1406_0359_gb300 import binding

    op = make_op(small, "fp32")
    L = binding.lib()
    assert L.purify_op_set_prior(op.h, 2, 10) == -1
    assert L.purify_op_set_prior(op.h, 1, 0) == -1
    assert L.purify_op_set_prior(op.h, 0, 0) == 0  # back to the l1 prior
    op.close()
