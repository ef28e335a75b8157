"""Pins for the oracle's proximity operators, CG and SDMM (Algorithm 1)."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize, minimize_scalar

from oracle import prox, sara
from oracle import sdmm as S
from oracle.cg import cg
from tests._tiny import tiny_problem


# ---------------------------------------------------------------- proxes (7)
@pytest.mark.parametrize("seed", range(5))
def test_soft_threshold_solves_eq7(seed):
    rng = np.random.default_rng(seed)
    for v, tau in zip(rng.normal(0, 2, 20), rng.uniform(0, 2, 20)):
        r = minimize_scalar(lambda z: tau * abs(z) + 0.5 * (v - z) ** 2,
                            bounds=(-10, 10), method="bounded", options={"xatol": 1e-12})
        assert prox.soft_threshold(np.array(v), tau) == pytest.approx(r.x, abs=1e-7)
    assert prox.soft_threshold(np.array([2.0, -2.0]), 2.0).tolist() == [0.0, 0.0]


def test_positive_projection_solves_eq7():
    rng = np.random.default_rng(1)
    for v in rng.normal(0, 2, 20):
        r = minimize_scalar(lambda z: 0.5 * (v - z) ** 2, bounds=(0, 10), method="bounded",
                            options={"xatol": 1e-12})
        assert prox.proj_positive(np.array(v)) == pytest.approx(r.x, abs=1e-7)


@pytest.mark.parametrize("seed", range(4))
def test_ball_projection_solves_eq7(seed):
    rng = np.random.default_rng(seed)
    y = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    v = y + rng.standard_normal(3) * 2 + 1j * rng.standard_normal(3)
    eps = 0.7
    to_c = lambda z: z[:3] + 1j * z[3:]
    res = minimize(lambda z: 0.5 * np.sum(np.abs(v - to_c(z)) ** 2),
                   np.concatenate([y.real, y.imag]), method="SLSQP",
                   constraints=[{"type": "ineq", "fun": lambda z: eps ** 2 - np.sum(np.abs(to_c(z) - y) ** 2)}],
                   options={"ftol": 1e-14, "maxiter": 500})
    p = prox.proj_l2_ball(v, y, eps)
    assert np.max(np.abs(p - to_c(res.x))) < 1e-5
    inside = y + 0.1 * (v - y) / np.linalg.norm(v - y)
    assert np.array_equal(prox.proj_l2_ball(inside, y, eps), inside)


def test_projections_firmly_nonexpansive():
    rng = np.random.default_rng(7)
    y = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    for _ in range(20):
        a = rng.standard_normal(50) * 3 + 1j * rng.standard_normal(50)
        b = rng.standard_normal(50) * 3 + 1j * rng.standard_normal(50)
        for P in (lambda v: prox.proj_l2_ball(v, y, 2.0),):
            pa, pb = P(a), P(b)
            lhs = np.sum(np.abs(pa - pb) ** 2)
            rhs = np.real(np.vdot(pa - pb, a - b))
            assert lhs <= rhs + 1e-12
        ra, rb = a.real, b.real
        for P in (prox.proj_positive, lambda v: prox.soft_threshold(v, 0.3)):
            pa, pb = P(ra), P(rb)
            assert np.sum((pa - pb) ** 2) <= np.sum((pa - pb) * (ra - rb)) + 1e-12


# ---------------------------------------------------------------- CG (step 5)
def test_cg_matches_dense_solve():
    T = tiny_problem()
    dop, nu = T["dop"], T["nu"]
    n = T["n"]
    A = nu * nu * np.real(T["Phi"].conj().T @ T["Phi"]) + 2.0 * np.eye(n * n)
    b = np.random.default_rng(0).standard_normal(n * n)
    ref = np.linalg.solve(A, b).reshape(n, n)
    Q = lambda v: nu * nu * dop.gram_real(v) + 2.0 * v
    x = cg(Q, b.reshape(n, n), np.zeros((n, n)), 60)
    assert np.max(np.abs(x - ref)) < 1e-10 * np.max(np.abs(ref))
    # warm start at the solution stays there
    x2 = cg(Q, b.reshape(n, n), ref, 5)
    assert np.max(np.abs(x2 - ref)) < 1e-12 * np.max(np.abs(ref))


# ---------------------------------------------------------------- SDMM
def test_composite_operator_identity():
    """sum_i L_i^H L_i = Psi Psi^H + I + Phi^H Phi = Phi^H Phi + 2I (Section 3)."""
    T = tiny_problem()
    x = np.random.default_rng(2).standard_normal((8, 8))
    lhs = T["dpsi"].synthesis(T["dpsi"].analysis(x)) + x + T["dop"].gram_real(x)
    rhs = T["dop"].gram_real(x) + 2.0 * x
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(rhs))


def test_feasible_zero_gives_zero():
    """eps >= ||y||: x = 0 is feasible and minimal, and SDMM never leaves it."""
    T = tiny_problem()
    w = np.ones(9 * 64)
    st = S.sdmm(T["dop"], T["dpsi"], T["y"], 1.01 * np.linalg.norm(T["y"]), 1e-3, w, 50, 10, T["nu"])
    assert np.all(st.x == 0.0)


def test_init_with_x0_is_a_fixed_point_of_the_first_update():
    """Steps 1-3 with z = 0 give sum_i x_i = Q x0, so step 5 returns x0."""
    T = tiny_problem()
    x0 = np.abs(np.random.default_rng(5).standard_normal((8, 8)))
    st = S.sdmm_init(T["dop"], T["dpsi"], x0, T["nu"])
    nu = T["nu"]
    Q = lambda v: nu * nu * T["dop"].gram_real(v) + 2.0 * v
    assert np.max(np.abs(st.xs - Q(x0))) < 1e-12 * np.max(np.abs(st.xs))


def _duality_gap(T, st, w, gamma):
    """Fenchel dual of problem (3) with the scaled ball (centre nu y, radius
    nu eps): maximise -Re<u3, nu y> - nu eps ||u3|| subject to |u1| <= w,
    u2 <= 0 and Psi u1 + u2 + nu Re Phi^H u3 = 0.  SDMM's scaled duals
    z_i / gamma give the candidate (u1 clipped to its box, u2 the nonpositive
    part of the balance); returns (relative gap, balance residual)."""
    nu = T["nu"]
    u1 = np.clip(st.z1 / gamma, -w, w)
    u3 = st.z3 / gamma
    s = T["dpsi"].synthesis(u1) + nu * T["dop"].phi_adj_real(u3)
    u2 = np.minimum(-s, 0.0)
    resid = np.linalg.norm(s + u2) / np.linalg.norm(T["dpsi"].synthesis(u1))
    dual = -np.real(np.vdot(u3, nu * T["y"])) - nu * T["eps"] * np.linalg.norm(u3)
    primal = float(np.sum(w * np.abs(T["dpsi"].analysis(st.x))))
    return (primal - dual) / primal, resid


@pytest.mark.slow
def test_sdmm_reaches_the_optimum_of_problem_3():
    """Algorithm 1 (oracle) closes the convex duality gap of problem (3):
    a certificate of optimality that does not rely on SDMM's own steps."""
    T = tiny_problem()
    w = np.random.default_rng(1).uniform(0.5, 1.5, 9 * 64)
    gamma = 10.0 * S.default_gamma(T["dop"], T["dpsi"], T["y"], T["nu"])
    st = S.sdmm(T["dop"], T["dpsi"], T["y"], T["eps"], gamma, w, 1500, 20, T["nu"])
    gap, resid = _duality_gap(T, st, w, gamma)
    assert 0.0 <= gap < 1e-6
    assert resid < 1e-4
    assert np.linalg.norm(T["y"] - T["dop"].phi(st.x)) <= T["eps"] * (1 + 1e-6)
    assert st.x.min() >= -1e-6 * st.x.max()
    # fixed point of Algorithm 1: sum_i L_i^H z_i -> 0
    nu = T["nu"]
    bal = T["dpsi"].synthesis(st.z1) + st.z2 + nu * T["dop"].phi_adj_real(st.z3)
    assert np.linalg.norm(bal) < 1e-5 * np.linalg.norm(T["dpsi"].synthesis(st.z1))


def test_sdmm_reaches_the_optimum_with_the_db8_dictionary():
    """Section 4's BPDb8 analysis problem (Db8 basis alone): the same
    duality-gap certificate as for SARA closes."""
    T = tiny_problem(bases=(8,))
    w = np.ones(64)
    gamma = 10.0 * S.default_gamma(T["dop"], T["dpsi"], T["y"], T["nu"])
    st = S.sdmm(T["dop"], T["dpsi"], T["y"], T["eps"], gamma, w, 1500, 20, T["nu"])
    gap, resid = _duality_gap(T, st, w, gamma)
    assert -1e-8 < gap < 1e-6
    assert resid < 1e-6
    assert np.linalg.norm(T["y"] - T["dop"].phi(st.x)) <= T["eps"] * (1 + 1e-6)


def test_sdmm_reaches_the_optimum_with_the_dirac_dictionary():
    """Section 4's BP problem (Psi = I): min ||x||_1, x >= 0, in the ball.  Here
    the dual candidate can be made exactly feasible -- u1 + u2 = -s with
    |u1| <= w and u2 <= 0 needs s >= -w, so u3 = z3 / gamma is scaled down
    until it holds -- and weak duality bounds the gap from below by 0."""
    T = tiny_problem(bases=(0,))
    nu, w = T["nu"], np.ones(64)
    gamma = 100.0 * S.default_gamma(T["dop"], T["dpsi"], T["y"], nu)
    st = S.sdmm(T["dop"], T["dpsi"], T["y"], T["eps"], gamma, w, 5000, 20, nu)
    u3 = st.z3 / gamma
    s = (nu * T["dop"].phi_adj_real(u3)).ravel()
    worst = float(np.max(-s / w))
    if worst > 1.0:
        u3 = u3 / worst
    dual = -np.real(np.vdot(u3, nu * T["y"])) - nu * T["eps"] * np.linalg.norm(u3)
    primal = float(np.sum(w * np.abs(st.x.ravel())))
    assert 0.0 <= (primal - dual) / primal < 1e-3
    assert np.linalg.norm(T["y"] - T["dop"].phi(st.x)) <= T["eps"] * (1 + 1e-4)
    assert st.x.min() >= -1e-6 * st.x.max()


def test_planted_sdmm_mistake_is_caught():
    """Dropping the dual update's sign (z <- z - (Lx - r)) stops SDMM reaching
    the optimum that the correct iteration reaches."""
    T = tiny_problem()
    w = np.ones(9 * 64)
    gamma = 10.0 * S.default_gamma(T["dop"], T["dpsi"], T["y"], T["nu"])
    good = S.sdmm(T["dop"], T["dpsi"], T["y"], T["eps"], gamma, w, 400, 20, T["nu"])
    st = S.sdmm_init(T["dop"], T["dpsi"], np.zeros((8, 8)), T["nu"])
    nu = T["nu"]
    Q = lambda v: nu * nu * T["dop"].gram_real(v) + 2.0 * v
    for _ in range(400):
        st.x = cg(Q, st.xs, st.x, 20)
        a1 = T["dpsi"].analysis(st.x)
        r1 = prox.soft_threshold(a1 + st.z1, gamma * w)
        st.z1 = st.z1 - (a1 - r1)  # planted sign error
        v2 = st.x + st.z2
        r2 = prox.proj_positive(v2)
        st.z2 = v2 - r2
        v3 = nu * T["dop"].phi(st.x) + st.z3
        r3 = prox.proj_l2_ball(v3, nu * T["y"], nu * T["eps"])
        st.z3 = v3 - r3
        st.xs = T["dpsi"].synthesis(r1 - st.z1) + (r2 - st.z2) + nu * T["dop"].phi_adj_real(r3 - st.z3)
    f_good = np.sum(np.abs(T["dpsi"].analysis(good.x)))
    f_bad = np.sum(np.abs(T["dpsi"].analysis(st.x)))
    feas_bad = np.linalg.norm(T["y"] - T["dop"].phi(st.x)) <= T["eps"] * 1.01
    assert not (feas_bad and abs(f_bad - f_good) < 1e-3 * f_good)


def test_reweighting_rule():
    alpha = np.array([0.0, 1.0, -3.0, 1e-9])
    d = S.delta_schedule(alpha, 1)
    assert d == pytest.approx(np.std(alpha))
    assert S.delta_schedule(alpha, 3) == pytest.approx(0.01 * np.std(alpha))
    assert S.delta_schedule(np.zeros(4), 1) == 1.0
    w = S.reweight(alpha, 0.5)
    assert w[0] == 1.0 and np.all((w > 0) & (w <= 1.0))
    assert w[2] == pytest.approx(0.5 / 3.5)


# ------------------------------------------------ reweighting as majorise-minimise
# Section 2.2 replaces the l0 prior by a sequence of weighted l1 problems whose
# weights come from the previous solution.  With w_j = delta / (delta + |a_j|)
# each round minimises, over the feasible set of problem (3), the linearisation
# at the previous solution of the concave penalty P(x) = sum_j log(delta +
# |(Psi^H x)_j|) (up to the constant factor delta).  Its tangent majorises P,
# so at a fixed delta every round that is solved to optimality cannot increase
# P (Candes, Wakin & Boyd 2008).  The pin runs the oracle's own SARA loop with a
# constant delta (decay 1, delta_min = delta0), certifies each round's optimality
# against the weights of the round before, and checks that P never rises.
def _mm_rounds(rounds, iters, reweight=None, monkeypatch=None):
    T = tiny_problem()
    gamma = 10.0 * S.default_gamma(T["dop"], T["dpsi"], T["y"], T["nu"])
    x0 = S.sdmm(T["dop"], T["dpsi"], T["y"], T["eps"], gamma, np.ones(9 * 64), iters, 20, T["nu"]).x
    delta = float(np.std(T["dpsi"].analysis(x0)))
    if reweight is not None:
        monkeypatch.setattr(S, "reweight", reweight)
    _, sts = S.sara_solve(T["dop"], T["dpsi"], T["y"], T["eps"], gamma, iters, 20, T["nu"], rounds,
                          decay=1.0, delta0=delta, delta_min=delta)
    pen = [float(np.sum(np.log(delta + np.abs(T["dpsi"].analysis(st.x))))) for st in sts]
    return T, gamma, delta, sts, np.array(pen)


@pytest.mark.slow
def test_reweighted_rounds_descend_the_log_penalty():
    T, gamma, delta, sts, pen = _mm_rounds(3, 1500)
    assert np.all(np.diff(pen) < 1e-7 * np.abs(pen[0]))  # P never rises
    assert pen[1] < pen[0] - 1e-3  # the first reweighting makes real progress
    for k in range(1, len(sts)):
        # round k is optimal for the weights taken from round k - 1's solution
        w = S.reweight(T["dpsi"].analysis(sts[k - 1].x), delta)
        gap, resid = _duality_gap(T, sts[k], w, gamma)
        assert abs(gap) < 1e-7 and resid < 1e-6
        assert np.linalg.norm(T["y"] - T["dop"].phi(sts[k].x)) <= T["eps"] * (1 + 1e-6)


@pytest.mark.slow
@pytest.mark.parametrize("plant", ["signed", "inverted", "squared"])
def test_planted_reweighting_mistakes_break_the_descent(plant, monkeypatch):
    """Plausible slips in the weight rule: the sign of the coefficient kept
    (no absolute value), the weight inverted, the denominator squared.  Each
    lets the log-penalty rise between rounds, which the pin above forbids."""
    bad = {"signed": lambda a, d: d / (d + a),
           "inverted": lambda a, d: (d + np.abs(a)) / d,
           "squared": lambda a, d: d / (d + np.abs(a)) ** 2}[plant]
    _, _, _, _, pen = _mm_rounds(3, 1500, bad, monkeypatch)
    assert np.max(np.diff(pen)) > 1e-3


@pytest.mark.slow
def test_stale_reweighting_coefficients_fail_the_certificate(monkeypatch):
    """Weights computed once from the first solution and reused (the wrong
    round's coefficients) leave later rounds optimal for stale weights: the
    certificate against the previous round's weights no longer closes."""
    rule = S.reweight
    first = {}

    def stale(a, d):
        first.setdefault("a", np.array(a, copy=True))
        return rule(first["a"], d)

    T, gamma, delta, sts, _ = _mm_rounds(2, 1500, stale, monkeypatch)
    w = rule(T["dpsi"].analysis(sts[1].x), delta)
    gap, _ = _duality_gap(T, sts[2], w, gamma)
    assert abs(gap) > 1e-5


def test_sara_outer_loop_runs_and_is_feasible():
    T = tiny_problem()
    gamma = 10.0 * S.default_gamma(T["dop"], T["dpsi"], T["y"], T["nu"])
    x, rounds = S.sara_solve(T["dop"], T["dpsi"], T["y"], T["eps"], gamma, 300, 20, T["nu"], 2)
    assert len(rounds) == 3
    assert np.linalg.norm(T["y"] - T["dop"].phi(x)) <= T["eps"] * 1.01
    assert x.min() >= -1e-6


# ---------------------------------------------------------------- R blocks (Eq. 4-5)
def _split(M, R, seed=0):
    perm = np.random.default_rng(seed).permutation(M)
    return [np.sort(perm[i::R]) for i in range(R)]


def test_single_block_equals_unblocked():
    T = tiny_problem()
    w = np.ones(9 * 64)
    g = 10.0 * S.default_gamma(T["dop"], T["dpsi"], T["y"], T["nu"])
    a = S.sdmm(T["dop"], T["dpsi"], T["y"], T["eps"], g, w, 40, 10, T["nu"])
    b = S.sdmm(T["dop"], T["dpsi"], T["y"], T["eps"], g, w, 40, 10, T["nu"],
               blocks=([np.arange(T["M"])], [T["eps"]]))
    assert np.array_equal(a.x, b.x)


def test_blocks_each_feasible_zero():
    T = tiny_problem()
    idx = _split(T["M"], 3)
    radii = [1.01 * np.linalg.norm(T["y"][i]) for i in idx]
    st = S.sdmm(T["dop"], T["dpsi"], T["y"], T["eps"], 1e-3, np.ones(9 * 64), 30, 10, T["nu"],
                blocks=(idx, radii))
    assert np.all(st.x == 0.0)


@pytest.mark.slow
def test_blocked_sdmm_closes_duality_gap():
    """R = 3 blocks with eps_i = eps sqrt(M_i / M): the Fenchel dual now has one
    ball term per block, -sum_i (Re<u_i, nu y_i> + nu eps_i ||u_i||)."""
    T = tiny_problem()
    M, nu = T["M"], T["nu"]
    idx = _split(M, 3)
    radii = [T["eps"] * np.sqrt(len(i) / M) for i in idx]
    w = np.random.default_rng(1).uniform(0.5, 1.5, 9 * 64)
    gamma = 10.0 * S.default_gamma(T["dop"], T["dpsi"], T["y"], nu)
    st = S.sdmm(T["dop"], T["dpsi"], T["y"], T["eps"], gamma, w, 2000, 20, nu, blocks=(idx, radii))
    u1 = np.clip(st.z1 / gamma, -w, w)
    u3 = st.z3 / gamma
    s = T["dpsi"].synthesis(u1) + nu * T["dop"].phi_adj_real(u3)
    u2 = np.minimum(-s, 0.0)
    resid = np.linalg.norm(s + u2) / np.linalg.norm(T["dpsi"].synthesis(u1))
    dual = -sum(np.real(np.vdot(u3[i], nu * T["y"][i])) + nu * e * np.linalg.norm(u3[i]) for i, e in zip(idx, radii))
    primal = float(np.sum(w * np.abs(T["dpsi"].analysis(st.x))))
    # weak duality up to the residual infeasibility of both iterates
    assert -1e-9 <= (primal - dual) / primal < 1e-5
    assert resid < 1e-3
    for i, e in zip(idx, radii):
        assert np.linalg.norm(T["y"][i] - T["dop"].phi(st.x)[i]) <= e * (1 + 1e-5)
