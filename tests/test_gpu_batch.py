"""Batched solver (many uneven instances, one launch per pass per image side,
one graph per iteration) against each instance's own solve and the oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import sdmm as osdmm
from paper_1406_0359_gb300 import synth
from tests._gpu import host, measured_problem, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu

# uneven instances: image side, visibility count, seed
MIX = [(128, 9000, 21), (64, 3000, 22), (256, 60000, 23), (128, 40000, 24), (64, 9000, 25), (256, 120000, 26),
       (128, 20000, 27)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()


def _instances(prec):
    from paper_1406_0359_gb300.binding import Operator

    out = []
    for n, M, seed in MIX:
        P = measured_problem(n, M, seed)
        op = Operator(torch.as_tensor(P["uv"]).cuda(), n, 3, prec)
        out.append((P, op, to_dev(P["y"], prec)))
    return out


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-11)])
def test_batched_instances_equal_their_solo_solves(prec, tol):
    from paper_1406_0359_gb300.binding import batch_solve

    inst = _instances(prec)
    kw = dict(t_max=12, cg_iters=8, n_reweight=1)
    solo = [op.solve(y, P["eps"], **kw) for P, op, y in inst]
    res = batch_solve([op for _, op, _ in inst], [y for _, _, y in inst], [P["eps"] for P, _, _ in inst], **kw)
    for a, b in zip(res, solo):
        assert a.stats["iterations"] == b.stats["iterations"] == 24
        assert a.stats["nu"] == pytest.approx(b.stats["nu"], rel=1e-12)
        assert rel(host(a.x), host(b.x)) < tol
        assert a.stats["objective"] == pytest.approx(b.stats["objective"], rel=10 * tol)
    for _, op, _ in inst:
        op.close()


def test_batched_instance_matches_oracle():
    from paper_1406_0359_gb300.binding import Operator, batch_solve

    P = measured_problem(64, 4096, 1)
    psi = osdmm.SaraDictionary(3)
    nu = 1.0 / math.sqrt(osdmm.operator_norm_sq(P["op"], 30))
    gamma = osdmm.default_gamma(P["op"], psi, P["y"], nu)
    x_ref, _ = osdmm.sara_solve(P["op"], psi, P["y"], P["eps"], gamma, 20, 10, nu, 1)
    others = _instances("fp32")[:3]
    op = Operator(torch.as_tensor(P["uv"]).cuda(), 64, 3, "fp32")
    ops = [op] + [o for _, o, _ in others]
    ys = [to_dev(P["y"], "fp32")] + [y for _, _, y in others]
    eps = [P["eps"]] + [Q["eps"] for Q, _, _ in others]
    res = batch_solve(ops, ys, eps, t_max=20, cg_iters=10, n_reweight=1, gamma=[gamma, 0, 0, 0], nu=[nu, 0, 0, 0])
    assert rel(host(res[0].x), x_ref) < 1e-3


def test_batch_refuses_what_it_cannot_group():
    from paper_1406_0359_gb300.binding import PurifyError, batch_solve

    inst = _instances("fp32")[:2]
    ops, ys = [o for _, o, _ in inst], [y for _, _, y in inst]
    eps = [P["eps"] for P, _, _ in inst]
    with pytest.raises(PurifyError):
        batch_solve(ops, ys, eps, t_max=3, cg_iters=2, xi=1e-3)
    with pytest.raises(PurifyError):
        batch_solve([ops[0], ops[0]], [ys[0], ys[0]], eps, t_max=3, cg_iters=2)
