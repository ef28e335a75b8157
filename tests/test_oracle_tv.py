"""Pins for the oracle's TV prior (Section 4's TV and RWTV): the discrete
operators, the TV proximity operator (Eq. 7) and SDMM (Algorithm 1) with the
TV block, each against closed forms, an exact 1-D solver, weak duality or a
duality-gap certificate."""
import math

import numpy as np
import pytest
from scipy.optimize import lsq_linear

from oracle import tv as TV
from tests._tiny import tiny_problem


def test_div_is_the_negative_adjoint_of_grad():
    rng = np.random.default_rng(0)
    for n in (2, 3, 8):
        x = rng.standard_normal((n, n))
        p = rng.standard_normal((2, n, n))
        assert np.sum(TV.grad(x) * p) == pytest.approx(-np.sum(x * TV.div(p)), abs=1e-12)


def test_grad_and_tv_closed_forms():
    n = 5
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    g = TV.grad(i.astype(float))  # ramp down the rows
    assert np.all(g[0, :-1] == 1.0) and np.all(g[0, -1] == 0.0) and np.all(g[1] == 0.0)
    assert TV.tv(np.full((n, n), 3.0)) == 0.0
    step = (i >= 2).astype(float)  # one unit jump in every column
    assert TV.tv(step) == pytest.approx(n)
    # x = i + j: (1, 1) inside, (0, 1) on the last row, (1, 0) on the last column, 0 at the corner
    assert TV.tv((i + j).astype(float)) == pytest.approx((n - 1) ** 2 * math.sqrt(2) + 2 * (n - 1))
    w = np.arange(1, n * n + 1, dtype=float).reshape(n, n)
    assert TV.tv(step, w) == pytest.approx(np.sum(w[1]))


@pytest.mark.parametrize("seed", range(3))
def test_tv_prox_closes_its_duality_gap(seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((8, 8))
    w = rng.uniform(0.5, 1.5, (8, 8))
    lam = 0.3
    x, q = TV.tv_prox(v, lam, w, 60000)
    assert np.all(TV.magnitude(q) <= lam * w * (1 + 1e-12))
    gap = TV.prox_duality_gap(v, lam, w, x, q)
    assert -1e-12 <= gap < 1e-9 * np.sum(v ** 2)
    # weak duality for an arbitrary feasible dual and primal
    q2 = TV.project(rng.standard_normal((2, 8, 8)), lam * w)
    assert TV.prox_duality_gap(v, lam, w, v + TV.div(q2) + 0.1, q2) > 0


def _prox_1d(v, lam_w):
    """Exact 1-D TV prox of one column: x = v - D^T u with the box-constrained
    least squares min |D^T u - v| over |u_i| <= lam w_i (library solver)."""
    n = v.size
    D = np.zeros((n - 1, n))
    D[np.arange(n - 1), np.arange(n - 1)] = -1.0
    D[np.arange(n - 1), np.arange(1, n)] = 1.0
    r = lsq_linear(D.T, v, bounds=(-lam_w, lam_w), tol=1e-14, lsmr_tol="auto", max_iter=10000)
    return v - D.T @ r.x


def test_tv_prox_of_column_constant_images_is_the_1d_prox():
    """v and w constant along each row: the prox is too, its second
    differences vanish, and each column solves the 1-D TV prox exactly."""
    rng = np.random.default_rng(5)
    n, lam = 8, 0.4
    f = rng.standard_normal(n) * 2
    wr = rng.uniform(0.5, 1.5, n)
    v = np.repeat(f[:, None], n, axis=1)
    w = np.repeat(wr[:, None], n, axis=1)
    x, _ = TV.tv_prox(v, lam, w, 6000)
    ref = _prox_1d(f, lam * wr[:-1])
    assert np.max(np.abs(x - ref[:, None])) < 1e-8


def test_tv_prox_limits():
    rng = np.random.default_rng(2)
    c = np.full((6, 6), 1.7)
    x, q = TV.tv_prox(c, 5.0, 1.0, 50)
    assert np.array_equal(x, c) and not np.any(q)
    v = rng.standard_normal((6, 6))
    x, _ = TV.tv_prox(v, 1e3, 1.0, 3000)  # the bound never binds: the constant of least squares
    assert np.max(np.abs(x - v.mean())) < 1e-9
    x, _ = TV.tv_prox(v, 0.0, 1.0, 10)
    assert np.array_equal(x, v)


@pytest.mark.parametrize("plant", ["anisotropic", "div_sign"])
def test_planted_tv_prox_mistakes_fail_the_gap(plant, monkeypatch):
    rng = np.random.default_rng(3)
    v = rng.standard_normal((8, 8))
    lam, w = 0.3, np.ones((8, 8))
    if plant == "anisotropic":
        monkeypatch.setattr(TV, "project", lambda q, b: np.clip(q, -b, b))
        x, q = TV.tv_prox(v, lam, w, 4000)
        monkeypatch.undo()
    else:
        real_div = TV.div
        monkeypatch.setattr(TV, "div", lambda p: -real_div(p))
        x, q = TV.tv_prox(v, lam, w, 400)
        monkeypatch.undo()
    q = TV.project(q, lam * w)
    assert TV.prox_duality_gap(v, lam, w, x, q) > 1e-4


def _tv_duality_gap(T, st, w, gamma):
    """Fenchel dual of the TV problem with the scaled ball: maximise
    -Re<u3, nu y> - nu eps ||u3|| subject to -div q + u2 + nu Re Phi^H u3 = 0,
    |q| <= w, u2 <= 0.  SDMM's duals give the candidate: u1 = z1 / gamma =
    -div(q_prox / gamma) exactly (the prox's own dual), u3 = z3 / gamma, u2
    the nonpositive part of the balance.  Returns (relative gap, balance
    residual)."""
    nu = T["nu"]
    qd = st.q / gamma
    assert np.all(TV.magnitude(qd) <= w * (1 + 1e-9))
    u1 = -TV.div(qd)
    u3 = st.z3 / gamma
    s = u1 + nu * T["dop"].phi_adj_real(u3)
    u2 = np.minimum(-s, 0.0)
    resid = np.linalg.norm(s + u2) / np.linalg.norm(u1)
    dual = -np.real(np.vdot(u3, nu * T["y"])) - nu * T["eps"] * np.linalg.norm(u3)
    primal = TV.tv(st.x, w)
    return (primal - dual) / primal, resid


@pytest.mark.slow
def test_tv_sdmm_reaches_the_optimum():
    T = tiny_problem()
    w = np.random.default_rng(4).uniform(0.5, 1.5, (8, 8))
    gamma = 10.0 * TV.tv_default_gamma(T["dop"], T["y"], T["nu"])
    st = TV.tv_sdmm(T["dop"], T["y"], T["eps"], gamma, w, 1500, 20, T["nu"], 30)
    gap, resid = _tv_duality_gap(T, st, w, gamma)
    assert -1e-9 <= gap < 1e-6
    assert resid < 1e-5
    assert np.linalg.norm(T["y"] - T["dop"].phi(st.x)) <= T["eps"] * (1 + 1e-6)
    assert st.x.min() >= -1e-6 * st.x.max()


@pytest.mark.slow
def test_tv_sdmm_with_a_planted_dual_sign_error_misses_the_optimum():
    T = tiny_problem()
    w = np.ones((8, 8))
    gamma = 10.0 * TV.tv_default_gamma(T["dop"], T["y"], T["nu"])
    good = TV.tv_sdmm(T["dop"], T["y"], T["eps"], gamma, w, 600, 20, T["nu"], 30)
    real = TV.tv_prox

    def bad_prox(v, lam, ww, iters, q0=None):  # returns v - div q: the dual's sign flipped
        x, q = real(v, lam, ww, iters, q0)
        return 2 * v - x, q

    TV.tv_prox = bad_prox
    try:
        bad = TV.tv_sdmm(T["dop"], T["y"], T["eps"], gamma, w, 600, 20, T["nu"], 30)
    finally:
        TV.tv_prox = real
    f_good, f_bad = TV.tv(good.x, w), TV.tv(bad.x, w)
    feas_bad = np.linalg.norm(T["y"] - T["dop"].phi(bad.x)) <= T["eps"] * 1.01
    assert not (feas_bad and abs(f_bad - f_good) < 1e-3 * f_good)


@pytest.mark.slow
def test_rwtv_rounds_descend_the_log_penalty():
    """RWTV at a fixed delta is majorise-minimise on sum_i log(delta + |grad x|_i):
    every round, certified optimal for the previous round's weights, must not
    raise it."""
    T = tiny_problem()
    gamma = 10.0 * TV.tv_default_gamma(T["dop"], T["y"], T["nu"])
    x0 = TV.tv_sdmm(T["dop"], T["y"], T["eps"], gamma, np.ones((8, 8)), 1500, 20, T["nu"], 30).x
    delta = float(np.std(TV.magnitude(TV.grad(x0))))
    _, sts = TV.tv_solve(T["dop"], T["y"], T["eps"], gamma, 1500, 20, T["nu"], 30, 3, decay=1.0, delta0=delta,
                         delta_min=delta)
    pen = np.array([np.sum(np.log(delta + TV.magnitude(TV.grad(st.x)))) for st in sts])
    assert np.all(np.diff(pen) < 1e-7 * abs(pen[0]))
    assert pen[1] < pen[0] - 1e-3
    for k in range(1, len(sts)):
        w = TV.rwtv_weights(sts[k - 1].x, delta)
        gap, resid = _tv_duality_gap(T, sts[k], w, gamma)
        assert abs(gap) < 1e-6 and resid < 1e-5
