"""GPU SDMM / SARA solver parity against the FP64 oracle (fixed iteration counts)."""
import math

import numpy as np
import pytest
import torch

from oracle import sdmm as osdmm
from oracle import simulate
from paper_1406_0359_gb300 import synth
from tests._gpu import host, measured_problem, need_gpu, rel, to_dev

pytestmark = pytest.mark.gpu

IMG_TOL = {"fp32": 1e-3, "fp64": 1e-9}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    need_gpu()


def make_op(P, levels, prec):
    from paper_1406_0359_gb300.binding import Operator

    return Operator(torch.as_tensor(P["uv"]).cuda(), P["n"], levels, prec)


@pytest.fixture(scope="module")
def small():
    P = measured_problem(64, 4096, 1)
    psi = osdmm.SaraDictionary(3)
    nu = 1.0 / math.sqrt(osdmm.operator_norm_sq(P["op"], 30))
    gamma = osdmm.default_gamma(P["op"], psi, P["y"], nu)
    P.update(psi=psi, nu=nu, gamma=gamma, levels=3)
    return P


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_auto_nu_and_gamma_match_oracle(small, prec):
    op = make_op(small, 3, prec)
    res = op.solve(to_dev(small["y"], prec), small["eps"], t_max=1, cg_iters=1, gram=0)
    tol = 1e-5 if prec == "fp32" else 1e-10
    assert res.stats["nu"] == pytest.approx(small["nu"], rel=tol)
    assert res.stats["gamma"] == pytest.approx(small["gamma"], rel=tol)


@pytest.mark.parametrize("prec,gram", [("fp32", 0), ("fp32", 1), ("fp64", 0), ("fp64", 1)])
@pytest.mark.parametrize("use_graph", [True, False])
def test_sara_solve_matches_oracle(small, prec, gram, use_graph):
    """Fixed-count SARA solve.  With gram = 1 the CG operator is the exact
    normal operator (PSF convolution) while the oracle applies the NUFFT's;
    they differ by the NUFFT error (~1e-7), so FP64 is held to 1e-5 there."""
    T, cg_iters, n_rw = 30, 10, 1
    x_ref, rounds = osdmm.sara_solve(small["op"], small["psi"], small["y"], small["eps"], small["gamma"], T,
                                     cg_iters, small["nu"], n_rw)
    op = make_op(small, 3, prec)
    res = op.solve(to_dev(small["y"], prec), small["eps"], t_max=T, cg_iters=cg_iters, n_reweight=n_rw,
                   gamma=small["gamma"], nu=small["nu"], use_graph=use_graph, gram=gram)
    xg = host(res.x)
    tol = IMG_TOL[prec] if (gram == 0 or prec == "fp32") else 1e-5
    assert rel(xg, x_ref) < tol
    assert res.stats["iterations"] == T * (n_rw + 1)
    last = rounds[-1].history[-1]
    assert res.stats["objective"] == pytest.approx(last["objective"], rel=10 * tol)
    assert res.stats["residual"] == pytest.approx(last["residual"], rel=10 * tol)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_feasible_zero_stays_zero(small, prec):
    op = make_op(small, 3, prec)
    eps = 1.01 * float(np.linalg.norm(small["y"]))
    res = op.solve(to_dev(small["y"], prec), eps, t_max=10, cg_iters=5, gamma=small["gamma"], nu=small["nu"])
    assert np.all(host(res.x) == 0.0)


def test_halting_rule_reports_status(small):
    from paper_1406_0359_gb300.binding import PurifyError

    op = make_op(small, 3, "fp32")
    res = op.solve(to_dev(small["y"], "fp32"), small["eps"], t_max=5, cg_iters=5, gamma=small["gamma"],
                   nu=small["nu"], xi=1e-12)
    assert res.status == -5 and res.stats["converged"] == 0
    res2 = op.solve(to_dev(small["y"], "fp32"), small["eps"], t_max=400, cg_iters=10, gamma=small["gamma"],
                    nu=small["nu"], xi=1e-3)
    assert res2.status in (0, -5)
    if res2.status == 0:
        assert res2.stats["iterations"] < 400 and res2.stats["converged"] == 1
    with pytest.raises(PurifyError):
        op.solve(to_dev(small["y"], "fp32"), -1.0)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_small_config_matches_oracle(prec):
    """64^2 sky, 4096 uv points, 3 levels, 200 SDMM iterations x 10 CG steps,
    3 reweighting rounds: final image within 1e-3 (FP32) and SNR within 0.05 dB."""
    w = synth.WORKLOADS["small_64"]
    P = measured_problem(w.n, w.M, w.seed, w.n_blobs, w.n_points)
    psi = osdmm.SaraDictionary(w.levels)
    nu = 1.0 / math.sqrt(osdmm.operator_norm_sq(P["op"], 30))
    gamma = osdmm.default_gamma(P["op"], psi, P["y"], nu)
    x_ref, _ = osdmm.sara_solve(P["op"], psi, P["y"], P["eps"], gamma, w.t_max, w.cg_iters, nu, w.n_reweight)
    op = make_op(P, w.levels, prec)
    res = op.solve(to_dev(P["y"], prec), P["eps"], t_max=w.t_max, cg_iters=w.cg_iters, n_reweight=w.n_reweight,
                   gamma=gamma, nu=nu, gram=0 if prec == "fp64" else -1)
    xg = host(res.x)
    assert rel(xg, x_ref) < IMG_TOL[prec]
    assert abs(simulate.snr_db(P["x_true"], xg) - simulate.snr_db(P["x_true"], x_ref)) < 0.05


def test_full_size_sara_and_fp32_solve_against_references():
    """1024^2 sky, 4,194,304 uv points, 4 levels (the bench workload): Psi^H
    and Psi against the oracle over the whole image, and three SDMM
    iterations of the FP32 path (graph, convolution-form CG) against the same
    iterations in FP64 on the GPU (NUFFT-form CG)."""
    from oracle import sara as osara
    from paper_1406_0359_gb300.binding import Operator

    w = synth.WORKLOADS["large_1024"]
    n, M, L = w.n, w.M, w.levels
    uv = synth.uv_coverage(M, n, w.seed)
    x = synth.sky(n, w.seed, w.n_blobs, w.n_points)
    op = Operator(torch.as_tensor(uv).cuda(), n, L, "fp32")
    c = op.sara_fwd(to_dev(x, "fp32"))
    c_ref = osara.analysis(x, L)
    assert rel(host(c), c_ref) < 1e-5
    assert rel(host(op.sara_adj(c)), osara.synthesis(c_ref, L)) < 1e-5
    y = op.phi(to_dev(x, "fp32"))
    eps = 0.05 * float(torch.linalg.vector_norm(y))
    r32 = op.solve(y, eps, t_max=3, cg_iters=w.cg_iters)
    op64 = Operator(torch.as_tensor(uv).cuda(), n, L, "fp64")
    r64 = op64.solve(y.to(torch.complex128), eps, t_max=3, cg_iters=w.cg_iters, nu=r32.stats["nu"],
                     gamma=r32.stats["gamma"], gram=0, use_graph=False)
    assert rel(host(r32.x), host(r64.x)) < 1e-4
