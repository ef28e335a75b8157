"""Sub-dictionaries of SARA on the GPU (Section 4's BP = Dirac, BPDb8 = Db8,
other selections) against the oracle: Psi^H / Psi element by element and
fixed-count (reweighted) solves."""
import math

import numpy as np
import pytest
import torch

from oracle import sara as osara
from oracle import sdmm as osdmm
from paper_1406_0359_gb300 import synth
from tests._gpu import host, measured_problem, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu

MASKS = [0x001, 0x100, 0x101, 0x026, 0x1FE, 0x1FF]
TOL = {"fp32": 1e-5, "fp64": 1e-11}


def bases_of(mask):
    return tuple(k for k in range(9) if mask >> k & 1)


@pytest.fixture(scope="module")
def uv64():
    need_gpu()
    return synth.uv_coverage(2000, 64, 3)


def make_op(uv, n, levels, prec):
    from paper_1406_0359_gb300.binding import Operator

    return Operator(torch.as_tensor(uv).cuda(), n, levels, prec)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("mask", MASKS)
def test_sub_dictionary_analysis_and_synthesis_match_oracle(uv64, mask, prec):
    n, levels = 64, 3
    op = make_op(uv64, n, levels, prec)
    op.set_dictionary(mask)
    got_mask, q = op.dictionary()
    assert got_mask == mask and q == bin(mask).count("1")
    x = synth.random_image(n, 21)
    c = host(op.sara_fwd(to_dev(x, prec)))
    c_ref = osara.analysis(x, levels, bases_of(mask))
    assert c.shape == c_ref.shape
    assert rel(c, c_ref) < TOL[prec]
    d = np.random.default_rng(mask).standard_normal(c_ref.shape)
    xs = host(op.sara_adj(to_dev(d, prec)))
    assert rel(xs, osara.synthesis(d, levels, bases_of(mask))) < TOL[prec]


def test_bad_masks_rejected(uv64):
    from paper_1406_0359_gb300.binding import PurifyError

    op = make_op(uv64, 64, 3, "fp32")
    for bad in (0, 0x200, 0x3FF):
        with pytest.raises(PurifyError):
            op.set_dictionary(bad)
    assert op.dictionary() == (0x1FF, 9)


@pytest.fixture(scope="module")
def small():
    need_gpu()
    P = measured_problem(64, 4096, 1)
    P["nu"] = 1.0 / math.sqrt(osdmm.operator_norm_sq(P["op"], 30))
    return P


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-3), ("fp64", 1e-9)])
@pytest.mark.parametrize("mask,n_rw", [(0x001, 0), (0x001, 1), (0x100, 0), (0x100, 1), (0x101, 1)])
def test_prior_solves_match_oracle(small, mask, n_rw, prec, tol):
    """BP, RWBP, BPDb8, RWBPDb8 and a two-basis dictionary: fixed-count solves
    (30 iterations, 10 CG steps) against the oracle with the same dictionary."""
    psi = osdmm.SaraDictionary(3, bases_of(mask))
    gamma = osdmm.default_gamma(small["op"], psi, small["y"], small["nu"])
    T, cg = 30, 10
    x_ref, _ = osdmm.sara_solve(small["op"], psi, small["y"], small["eps"], gamma, T, cg, small["nu"], n_rw)
    op = make_op(small["uv"], 64, 3, prec)
    op.set_dictionary(mask)
    res = op.solve(to_dev(small["y"], prec), small["eps"], t_max=T, cg_iters=cg, n_reweight=n_rw, gamma=gamma,
                   nu=small["nu"], gram=0)
    assert rel(host(res.x), x_ref) < tol


def test_default_gamma_follows_the_dictionary(small):
    """The library's gamma rule uses the selected Psi^H."""
    psi = osdmm.SaraDictionary(3, (8,))
    gamma = osdmm.default_gamma(small["op"], psi, small["y"], small["nu"])
    op = make_op(small["uv"], 64, 3, "fp64")
    op.set_dictionary(0x100)
    res = op.solve(to_dev(small["y"], "fp64"), small["eps"], t_max=1, cg_iters=1, nu=small["nu"], gram=0)
    assert res.stats["gamma"] == pytest.approx(gamma, rel=1e-10)
