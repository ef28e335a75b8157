"""Total-variation prior for the same constrained problem (oracle, FP64, test infrastructure only).

Section 4 compares the l1 analysis problems with TV minimisation under the
same data constraint and positivity ("TV"), and with its reweighted version
("RWTV").  The paper gives neither the discrete TV nor how its proximity
operator is computed; readings:

* discrete isotropic TV with forward differences and a zero difference past
  the last row / column (Neumann boundary):
      (grad x)_1[i, j] = x[i+1, j] - x[i, j]  (0 on the last row),
      (grad x)_2[i, j] = x[i, j+1] - x[i, j]  (0 on the last column),
      TV_w(x) = sum_ij w_ij sqrt((grad x)_1[i, j]^2 + (grad x)_2[i, j]^2),
  with per-pixel weights w (w = 1 for TV; RWTV reweights them);
* div = -grad^T (the discrete divergence), so <grad x, p> = -<x, div p>;
* prox of lam TV_w (Eq. 7) through its dual: x = v + div q where q solves
      min over |q_ij| <= lam w_ij of  (1/2) || v + div q ||^2,
  by projected gradient q <- P(q + tau grad(v + div q)) with tau = 1/8
  (||div||^2 <= 8), a fixed number of steps from a given start q0;
* inside SDMM (Algorithm 1) the TV block is f_1 = gamma TV_w with L_1 = I, so
  the composite operator is still nu^2 Phi^H Phi + 2I; the TV prox takes
  `tv_iters` dual steps per SDMM iteration, warm-started from the previous
  iteration's dual (zero at the start of each round);
* RWTV: w_i = delta / (delta + |grad x_hat|_i) from the previous round's
  solution, delta from the same schedule as SARA's (sdmm.delta_schedule)
  applied to the gradient magnitudes.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .cg import cg
from .prox import proj_l2_ball, proj_positive
from .sdmm import delta_schedule

TAU = 1.0 / 8.0


def grad(x: np.ndarray) -> np.ndarray:
    """Forward differences, (2, n, n); zero past the last row / column."""
    g = np.zeros((2,) + x.shape)
    g[0, :-1, :] = x[1:, :] - x[:-1, :]
    g[1, :, :-1] = x[:, 1:] - x[:, :-1]
    return g


def div(p: np.ndarray) -> np.ndarray:
    """Discrete divergence, the negative adjoint of grad."""
    p1, p2 = p[0], p[1]
    d = np.zeros(p1.shape)
    d[0, :] += p1[0, :]
    d[1:-1, :] += p1[1:-1, :] - p1[:-2, :]
    d[-1, :] -= p1[-2, :]
    d[:, 0] += p2[:, 0]
    d[:, 1:-1] += p2[:, 1:-1] - p2[:, :-2]
    d[:, -1] -= p2[:, -2]
    return d


def magnitude(g: np.ndarray) -> np.ndarray:
    return np.sqrt(g[0] ** 2 + g[1] ** 2)


def tv(x: np.ndarray, w=1.0) -> float:
    """Weighted isotropic TV."""
    return float(np.sum(w * magnitude(grad(x))))


def project(q: np.ndarray, bound: np.ndarray) -> np.ndarray:
    """Pixelwise projection of the dual vectors onto |q_ij| <= bound_ij."""
    m = magnitude(q)
    s = np.where(m > bound, bound / np.where(m > 0, m, 1.0), 1.0)
    return q * s


def tv_prox(v: np.ndarray, lam: float, w, iters: int, q0=None):
    """prox of lam TV_w at v by `iters` projected-gradient steps on the dual
    from q0 (zero when None); returns (x, q)."""
    v = np.asarray(v, dtype=np.float64)
    bound = lam * np.broadcast_to(np.asarray(w, dtype=np.float64), v.shape)
    q = np.zeros((2,) + v.shape) if q0 is None else np.array(q0, dtype=np.float64, copy=True)
    for _ in range(iters):
        q = project(q + TAU * grad(v + div(q)), bound)
    return v + div(q), q


def prox_duality_gap(v, lam, w, x, q) -> float:
    """P(x) - D(q) for the prox problem: P(x) = |x - v|^2 / 2 + lam TV_w(x),
    D(q) = |v|^2 / 2 - |v + div q|^2 / 2 for |q| <= lam w (weak duality makes
    it >= 0; it is 0 exactly at the solution pair)."""
    P = 0.5 * float(np.sum((x - v) ** 2)) + lam * tv(x, w)
    D = 0.5 * float(np.sum(v ** 2)) - 0.5 * float(np.sum((v + div(q)) ** 2))
    return P - D


# ----------------------------------------------------------------- SDMM with the TV block
@dataclass
class TVState:
    x: np.ndarray
    z1: np.ndarray
    z2: np.ndarray
    z3: np.ndarray
    xs: np.ndarray
    q: np.ndarray  # the TV prox's dual, carried between iterations
    t: int = 0
    history: list = field(default_factory=list)


def tv_sdmm_init(op, x0: np.ndarray, nu: float) -> TVState:
    """Steps 1-3 of Algorithm 1 with L_1 = L_2 = I, L_3 = nu Phi."""
    r3 = nu * op.phi(x0)
    xs = 2.0 * x0 + nu * op.phi_adj_real(r3)
    z = np.zeros_like(x0, dtype=np.float64)
    return TVState(x=np.array(x0, dtype=np.float64, copy=True), z1=z.copy(), z2=z.copy(),
                   z3=np.zeros_like(r3), xs=xs, q=np.zeros((2,) + x0.shape))


def tv_sdmm_iteration(st: TVState, op, y, eps, gamma, w, cg_iters, nu, tv_iters) -> dict:
    """Steps 5-10 of Algorithm 1 for f_1 = gamma TV_w (L_1 = I), positivity and the ball."""

    def Q(v):  # sum_i L_i^H L_i = nu^2 Re Phi^H Phi + 2 I
        return nu * nu * op.gram_real(v) + 2.0 * v

    st.x = cg(Q, st.xs, st.x, cg_iters)
    xh = st.x
    # block 1: weighted TV
    v1 = xh + st.z1
    r1, st.q = tv_prox(v1, gamma, w, tv_iters, st.q)
    st.z1 = v1 - r1
    x1 = r1 - st.z1
    # block 2: positivity
    v2 = xh + st.z2
    r2 = proj_positive(v2)
    st.z2 = v2 - r2
    x2 = r2 - st.z2
    # block 3: data fidelity, the scaled ball
    phx = op.phi(xh)
    v3 = nu * phx + st.z3
    r3 = proj_l2_ball(v3, nu * y, nu * eps)
    st.z3 = v3 - r3
    x3 = nu * op.phi_adj_real(r3 - st.z3)
    st.xs = x1 + x2 + x3
    st.t += 1
    diag = {"objective": tv(xh, w), "residual": float(np.linalg.norm(y - phx))}
    st.history.append(diag)
    return diag


def tv_sdmm(op, y, eps, gamma, w, t_max, cg_iters, nu, tv_iters, x0=None) -> TVState:
    n = op.n
    st = tv_sdmm_init(op, np.zeros((n, n)) if x0 is None else x0, nu)
    for _ in range(t_max):
        tv_sdmm_iteration(st, op, y, eps, gamma, w, cg_iters, nu, tv_iters)
    return st


def tv_default_gamma(op, y, nu: float) -> float:
    """gamma = 1e-3 ||nu^2 Re Phi^H y||_inf (reading, as for the l1 prior with
    Psi = I)."""
    return 1e-3 * float(np.max(np.abs(nu * nu * op.phi_adj_real(y))))


def rwtv_weights(x: np.ndarray, delta: float) -> np.ndarray:
    """RWTV weights delta / (delta + |grad x|) per pixel."""
    return delta / (delta + magnitude(grad(x)))


def tv_solve(op, y, eps, gamma, t_max, cg_iters, nu, tv_iters, n_reweight, decay=0.1, delta0=None,
             delta_min=None, warm_start=True):
    """TV (n_reweight = 0) or RWTV: an unweighted solve followed by n_reweight
    reweighted ones.  Returns (x, list of per-round TVState)."""
    n = op.n
    w = np.ones((n, n))
    st = tv_sdmm(op, y, eps, gamma, w, t_max, cg_iters, nu, tv_iters)
    rounds = [st]
    g0 = magnitude(grad(st.x))
    for k in range(1, n_reweight + 1):
        delta = delta_schedule(g0, k, decay, delta0, delta_min)
        w = rwtv_weights(st.x, delta)
        st = tv_sdmm(op, y, eps, gamma, w, t_max, cg_iters, nu, tv_iters, st.x if warm_start else None)
        rounds.append(st)
    return st.x, rounds
