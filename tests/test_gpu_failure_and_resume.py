"""Failure detection and checkpoint / resume through the C-ABI.

No test here faults, traps or hangs the GPU.  A bounded device wait is made
to run out by arming an mbarrier for bytes that are never sent (the
library's self-test kernel, with a short spin budget); bad inputs are made on
the host (NaN in uv or y); a solve is stopped between SDMM iterations, saved
to host memory and resumed on a fresh operator; a request is cancelled
between iterations.
"""
import math

import numpy as np
import pytest
import torch

from oracle import sdmm as osdmm
from paper_1406_0359_gb300 import synth
from tests._gpu import host, measured_problem, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()


@pytest.fixture(scope="module")
def small():
    P = measured_problem(64, 4096, 1)
    psi = osdmm.SaraDictionary(3)
    nu = 1.0 / math.sqrt(osdmm.operator_norm_sq(P["op"], 30))
    gamma = osdmm.default_gamma(P["op"], psi, P["y"], nu)
    P.update(nu=nu, gamma=gamma)
    return P


def make_op(P, prec="fp32"):
    from paper_1406_0359_gb300.binding import Operator

    return Operator(torch.as_tensor(P["uv"]).cuda(), P["n"], 3, prec)


def test_bounded_wait_times_out_and_the_context_stays_usable(small):
    from paper_1406_0359_gb300 import binding

    binding.purify_set_wait_limit(2000)
    try:
        assert binding.purify_wait_selftest(True) == 0  # bytes delivered: the wait completes
        assert binding.purify_wait_selftest(False) == -4  # nothing sent: PURIFY_ERR_TIMEOUT
        assert "gave up" in binding.lib().purify_last_error().decode()
        assert binding.purify_wait_selftest(True) == 0
    finally:
        binding.purify_set_wait_limit(0)
    op = make_op(small)
    y = op.phi(to_dev(small["x_true"], "fp32"))
    assert rel(host(y), small["op"].phi(small["x_true"])) < 1e-5
    op.close()


def test_nonfinite_inputs_are_rejected(small):
    from paper_1406_0359_gb300.binding import Operator, PurifyError

    uv = np.array(small["uv"], copy=True)
    uv[17, 1] = np.nan
    with pytest.raises(PurifyError) as e:
        Operator(torch.as_tensor(uv).cuda(), 64, 3, "fp32")
    assert e.value.code == -1 and "non-finite" in str(e.value)
    op = make_op(small)
    y = np.array(small["y"], copy=True)
    y[5] = np.inf
    with pytest.raises(PurifyError) as e:
        op.solve(to_dev(y, "fp32"), small["eps"], t_max=3, cg_iters=3, gamma=small["gamma"], nu=small["nu"])
    assert e.value.code == -1 and "non-finite" in str(e.value)
    # the operator is still usable afterwards
    res = op.solve(to_dev(small["y"], "fp32"), small["eps"], t_max=3, cg_iters=3, gamma=small["gamma"],
                   nu=small["nu"])
    assert res.status == 0 and np.all(np.isfinite(host(res.x)))
    op.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-11)])
@pytest.mark.parametrize("stop", [13, 47])
def test_resumed_solve_matches_uninterrupted(small, prec, tol, stop):
    """T = 30 iterations per round and one reweighting (60 in all); the solve
    is stopped after `stop` iterations (inside round 0, inside round 1),
    saved, and resumed on a new operator built from the same inputs."""
    kw = dict(t_max=30, cg_iters=8, n_reweight=1, gamma=small["gamma"], nu=small["nu"])
    y = to_dev(small["y"], prec)
    op = make_op(small, prec)
    ref = op.solve(y, small["eps"], **kw)
    op.close()
    a = make_op(small, prec)
    a.solve_begin(y, small["eps"], **kw)
    assert not a.solve_step(stop)
    state = a.save_state()
    assert a.save_state() == state  # saving changes nothing
    a.close()
    b = make_op(small, prec)
    b.solve_begin(y, small["eps"], **kw)
    b.load_state(state)
    assert b.save_state() == state  # the round trip is exact
    while not b.solve_step(7):
        pass
    res = b.solve_end()
    b.close()
    assert res.stats["iterations"] == ref.stats["iterations"] == 60
    assert res.stats["rounds"] == 2
    assert rel(host(res.x), host(ref.x)) < tol
    assert res.stats["objective"] == pytest.approx(ref.stats["objective"], rel=10 * tol)


def test_checkpoint_of_another_operator_is_rejected(small):
    from paper_1406_0359_gb300.binding import Operator, PurifyError

    kw = dict(t_max=5, cg_iters=3, gamma=small["gamma"], nu=small["nu"])
    a = make_op(small)
    a.solve_begin(to_dev(small["y"], "fp32"), small["eps"], **kw)
    a.solve_step(2)
    state = a.save_state()
    a.close()
    uv = synth.uv_coverage(2048, 64, 9)
    b = Operator(torch.as_tensor(uv).cuda(), 64, 3, "fp32")
    b.solve_begin(torch.zeros(2048, dtype=torch.complex64, device="cuda"), 1.0, **kw)
    with pytest.raises(PurifyError):
        b.load_state(state)
    b.close()
