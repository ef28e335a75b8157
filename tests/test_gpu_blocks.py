"""R visibility blocks (Eq. 4-5) on the GPU against the oracle's blocked SDMM."""
import math

import numpy as np
import pytest
import torch

from oracle import sdmm as osdmm
from tests._gpu import host, measured_problem, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prob():
    need_gpu()
    P = measured_problem(64, 4096, 1)
    psi = osdmm.SaraDictionary(3)
    nu = 1.0 / math.sqrt(osdmm.operator_norm_sq(P["op"], 30))
    gamma = osdmm.default_gamma(P["op"], psi, P["y"], nu)
    R = 4
    bid = np.random.default_rng(5).integers(0, R, P["M"]).astype(np.int32)
    idx = [np.flatnonzero(bid == b) for b in range(R)]
    radii = [P["eps"] * math.sqrt(len(i) / P["M"]) * (0.9 + 0.1 * b) for b, i in enumerate(idx)]
    P.update(psi=psi, nu=nu, gamma=gamma, R=R, bid=bid, idx=idx, radii=radii)
    return P


def make_op(P, prec):
    from paper_1406_0359_gb300.binding import Operator

    return Operator(torch.as_tensor(P["uv"]).cuda(), P["n"], 3, prec)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-9)])
def test_blocked_solve_matches_oracle(prob, prec, tol):
    T, cg = 30, 10
    x_ref, rounds = osdmm.sara_solve(prob["op"], prob["psi"], prob["y"], prob["eps"], prob["gamma"], T, cg,
                                     prob["nu"], 1, blocks=(prob["idx"], prob["radii"]))
    op = make_op(prob, prec)
    op.set_blocks(prob["bid"], prob["R"])
    res = op.solve(to_dev(prob["y"], prec), prob["eps"], t_max=T, cg_iters=cg, n_reweight=1, gamma=prob["gamma"],
                   nu=prob["nu"], gram=0, eps_blocks=prob["radii"])
    assert rel(host(res.x), x_ref) < tol
    last = rounds[-1].history[-1]
    assert res.stats["residual"] == pytest.approx(last["residual"], rel=10 * tol)


def test_one_block_equals_default(prob):
    op = make_op(prob, "fp64")
    y = to_dev(prob["y"], "fp64")
    kw = dict(t_max=10, cg_iters=5, gamma=prob["gamma"], nu=prob["nu"], gram=0)
    a = host(op.solve(y, prob["eps"], **kw).x)
    op.set_blocks(np.zeros(prob["M"], np.int32), 1)
    b = host(op.solve(y, prob["eps"], **kw).x)
    assert rel(b, a) < 1e-12


def test_bad_block_ids_rejected(prob):
    from paper_1406_0359_gb300.binding import PurifyError

    op = make_op(prob, "fp32")
    bad = prob["bid"].copy()
    bad[7] = prob["R"]
    with pytest.raises(PurifyError):
        op.set_blocks(bad, prob["R"])
