"""An operator keeps its captured iteration graph across solves.  A repeated
solve with the same scalars replays it; any change of nu, gamma, eps, the CG
steps, the dictionary, the prior, the visibility blocks or the normal-operator
form must capture afresh.  Each case compares the reused operator with a fresh
one and with a solve without graph replay, within 1e-5 (gridding's atomic
additions make runs differ in rounding); every change moves the image by more
than 1e-4, so a stale graph would show."""
import numpy as np
import pytest
import torch

from tests._gpu import host, measured_problem, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prob():
    need_gpu()
    return measured_problem(64, 4000, 71)


def _fresh(P, setup=None):
    from paper_1406_0359_gb300.binding import Operator

    op = Operator(torch.as_tensor(P["uv"]).cuda(), 64, 3, "fp32")
    if setup:
        setup(op)
    return op


def _solve(op, P, **kw):
    kw = dict(dict(t_max=6, cg_iters=6, nu=1e-2, gamma=1e-3), **kw)
    return host(op.solve(to_dev(P["y"], "fp32"), P["eps"], **kw).x)


def test_repeated_solve_replays_the_same_graph(prob):
    op = _fresh(prob)
    a = _solve(op, prob)
    b = _solve(op, prob)
    assert rel(b, a) < 1e-5
    c = _solve(op, prob, use_graph=False)
    assert rel(c, a) < 1e-5
    op.close()


@pytest.mark.parametrize("change", ["nu", "gamma", "eps", "cg_iters"])
def test_changed_scalars_capture_again(prob, change):
    op = _fresh(prob)
    base = _solve(op, prob)  # the graph of the defaults
    kw = {"nu": dict(nu=2e-2), "gamma": dict(gamma=3e-3), "eps": {}, "cg_iters": dict(cg_iters=2)}[change]
    P2 = dict(prob, eps=prob["eps"] * 1.5) if change == "eps" else prob
    a = _solve(op, P2, **kw)
    fresh = _fresh(prob)
    b = _solve(fresh, P2, **kw)
    assert rel(a, b) < 1e-5
    assert rel(base, b) > 1e-4
    op.close()
    fresh.close()


@pytest.mark.parametrize("change", ["dictionary", "prior", "blocks", "nufft_form"])
def test_changed_structure_captures_again(prob, change):
    def setup(op):
        if change == "dictionary":
            op.set_dictionary(1 | (1 << 8))  # Dirac + Db8
        elif change == "prior":
            op.set_prior("tv", 7)
        elif change == "blocks":
            ids = (np.arange(prob["M"]) % 3).astype(np.int32)
            op.set_blocks(ids, 3)

    kw = dict(gram=0) if change == "nufft_form" else {}
    op = _fresh(prob)
    base = _solve(op, prob)  # the graph of the default structure
    setup(op)
    a = _solve(op, prob, **kw)
    fresh = _fresh(prob, setup)
    b = _solve(fresh, prob, **kw)
    assert rel(a, b) < 1e-5
    assert rel(_solve(fresh, prob, use_graph=False, **kw), b) < 1e-5
    if change != "nufft_form":  # the NUFFT form solves the same problem (NUFFT-level differences)
        assert rel(base, b) > 1e-4
    op.close()
    fresh.close()
