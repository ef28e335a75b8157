"""SDMM (Algorithm 1) and the SARA reweighting loop (oracle, FP64, test infrastructure only).

Problem (3): min ||W Psi^H x||_1 over x in R_+^N subject to ||y - Phi x|| <= eps,
written as (6) with S = 3 functions (one visibility block, R = 1):
    f_1 = ||W .||_1, L_1 = Psi^H;   f_2 = indicator of R_+^N, L_2 = I;
    f_3 = indicator of the eps-ball around y, L_3 = Phi.
Algorithm 1 then alternates the global update
    x_hat = (sum_i L_i^H L_i)^-1 sum_i x_i
(solved by conjugate gradient, step 5; the composite operator equals
Phi^H Phi + 2I because Psi Psi^H = I, Section 3) with, for every i,
    r_i = prox_{gamma f_i}(L_i x_hat + z_i),  z_i += L_i x_hat - r_i,
    x_i = L_i^H (r_i - z_i).
With the visibilities split into R blocks (Eq. 4) the data term becomes R
balls ||y_i - Phi_i x|| <= eps_i (Eq. 5), S = R + 2 functions, L_{i+2} = Phi_i
(Eq. 6); each block gets its own projection, and sum_i Phi_i^H Phi_i = Phi^H Phi
keeps the composite operator unchanged (Section 3).
Readings (the paper is silent): x is real, so L_3^H = Re Phi^H; inside the
solver Phi is scaled by nu = 1/||Phi||_2 together with the ball centres and
radii, which leaves problem (3) unchanged; the halting rule is
|f_t - f_{t-1}| < xi f_{t-1} together with ||y_i - Phi_i x_hat|| <= eps_i (1 + 1e-3)
for every block, f_t = ||W Psi^H x_hat||_1; xi = 0 never halts.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import sara as sara_mod
from .cg import cg


class SaraDictionary:
    """Psi^H / Psi pair for the SDMM blocks: the SARA dictionary at a fixed
    number of wavelet levels (sara.py), or one of its sub-dictionaries
    (`bases`: 0 = Dirac, K = DbK; Section 4's BP is (0,), BPDb8 is (8,)).  Any
    object with the same two methods (and a tight frame) can stand in, e.g. a
    dense matrix in tests."""

    def __init__(self, levels: int, bases=sara_mod.ALL_BASES):
        self.levels = levels
        self.bases = sara_mod._check(bases)

    def analysis(self, x):
        return sara_mod.analysis(x, self.levels, self.bases)

    def synthesis(self, c):
        return sara_mod.synthesis(c, self.levels, self.bases)
from .prox import proj_l2_ball, proj_positive, soft_threshold


def operator_norm_sq(op, iters: int = 30) -> float:
    """||Phi||_2^2 (restricted to real images) by power iteration on
    Re(Phi^H Phi), started from the all-ones image."""
    x = np.ones((op.n, op.n)) / op.n
    lam = 0.0
    for _ in range(iters):
        v = op.gram_real(x)
        lam = float(np.linalg.norm(v))
        x = v / lam
    return lam


def default_gamma(op, psi, y: np.ndarray, nu: float) -> float:
    """gamma = 1e-3 * ||Psi^H (nu^2 Re Phi^H y)||_inf (reading; Algorithm 1
    only asks gamma > 0)."""
    return 1e-3 * float(np.max(np.abs(psi.analysis(nu * nu * op.phi_adj_real(y)))))


@dataclass
class SDMMState:
    x: np.ndarray
    z1: np.ndarray
    z2: np.ndarray
    z3: np.ndarray
    xs: np.ndarray  # sum_i x_i
    t: int = 0
    history: list = field(default_factory=list)


def sdmm_init(op, psi, x0: np.ndarray, nu: float) -> SDMMState:
    """Steps 1-3 of Algorithm 1: z_i = 0, r_i = L_i x0, x_i = L_i^H r_i."""
    r1 = psi.analysis(x0)
    r2 = np.array(x0, copy=True)
    r3 = nu * op.phi(x0)
    xs = psi.synthesis(r1) + r2 + nu * op.phi_adj_real(r3)
    return SDMMState(
        x=np.array(x0, dtype=np.float64, copy=True),
        z1=np.zeros_like(r1),
        z2=np.zeros_like(r2),
        z3=np.zeros_like(r3),
        xs=xs,
    )


def _blocks(M, eps, blocks):
    """(index arrays, radii): one block of all visibilities unless given."""
    if blocks is None:
        return [np.arange(M)], [float(eps)]
    idx, radii = blocks
    return [np.asarray(i) for i in idx], [float(e) for e in radii]


def sdmm_iteration(st: SDMMState, op, psi, y, eps, gamma, w, cg_iters, nu, blocks=None) -> dict:
    """One pass of steps 5-10 of Algorithm 1 (in place); returns diagnostics.
    `blocks` = (list of index arrays, list of eps_i) for R > 1 (Eq. 4-5)."""

    def Q(v):  # sum_i L_i^H L_i = nu^2 Re Phi^H Phi + 2 I
        return nu * nu * op.gram_real(v) + 2.0 * v

    st.x = cg(Q, st.xs, st.x, cg_iters)
    xh = st.x
    # block 1: l1 on the SARA coefficients
    a1 = psi.analysis(xh)
    v1 = a1 + st.z1
    r1 = soft_threshold(v1, gamma * w)
    st.z1 = v1 - r1
    x1 = psi.synthesis(r1 - st.z1)
    # block 2: positivity
    v2 = xh + st.z2
    r2 = proj_positive(v2)
    st.z2 = v2 - r2
    x2 = r2 - st.z2
    # blocks 3..S: data fidelity, one scaled ball per visibility block
    phx = op.phi(xh)
    v3 = nu * phx + st.z3
    r3 = np.empty_like(v3)
    idx, radii = _blocks(op.M, eps, blocks)
    for ib, eb in zip(idx, radii):
        r3[ib] = proj_l2_ball(v3[ib], nu * y[ib], nu * eb)
    st.z3 = v3 - r3
    x3 = nu * op.phi_adj_real(r3 - st.z3)  # sum_i Phi_i^H (r_i - z_i)
    st.xs = x1 + x2 + x3
    st.t += 1
    diag = {
        "objective": float(np.sum(w * np.abs(a1))),
        "residual": float(np.linalg.norm(y - phx)),
        "block_residuals": [float(np.linalg.norm(y[ib] - phx[ib])) for ib in idx],
    }
    st.history.append(diag)
    return diag


def sdmm(op, psi, y, eps, gamma, w, t_max, cg_iters, nu, x0=None, xi=0.0, blocks=None):
    """Run Algorithm 1 for t_max iterations or until the halting rule fires."""
    n = op.n
    x0 = np.zeros((n, n)) if x0 is None else x0
    st = sdmm_init(op, psi, x0, nu)
    _, radii = _blocks(op.M, eps, blocks)
    prev = None
    for _ in range(t_max):
        d = sdmm_iteration(st, op, psi, y, eps, gamma, w, cg_iters, nu, blocks)
        if xi > 0.0 and prev is not None:
            rel = abs(d["objective"] - prev) / max(prev, 1e-300)
            feas = all(rb <= eb * (1.0 + 1e-3) for rb, eb in zip(d["block_residuals"], radii))
            if rel < xi and feas:
                break
        prev = d["objective"]
    return st


def delta_schedule(alpha0: np.ndarray, k: int, decay: float = 0.1, delta0=None, delta_min=None) -> float:
    """Reweighting parameter for round k >= 1 (reading; parity unpinned: the
    paper fixes no schedule, and no identity constrains one):
    delta_1 = std of the round-0 coefficients (or delta0 when given, 1 when
    the coefficients are all zero), delta_k = max(decay^(k-1) delta_1, delta_min),
    delta_min defaulting to 1e-4 delta_1."""
    d1 = float(delta0) if delta0 else float(np.std(alpha0))
    if d1 <= 0.0:
        d1 = 1.0
    dmin = float(delta_min) if delta_min else 1e-4 * d1
    return max(decay ** (k - 1) * d1, dmin)


def reweight(alpha: np.ndarray, delta: float) -> np.ndarray:
    """SARA weights w_j = delta / (delta + |alpha_j|) (Section 2.2: each round's
    weight on a coefficient falls off as the inverse of that coefficient's
    magnitude in the previous solution; delta keeps it finite).  Pinned as a
    majorise-minimise step: at fixed delta the rounds descend
    sum_j log(delta + |alpha_j|) (tests/test_oracle_solver.py)."""
    return delta / (delta + np.abs(alpha))


def sara_solve(op, psi, y, eps, gamma, t_max, cg_iters, nu, n_reweight,
               decay=0.1, delta0=None, delta_min=None, warm_start=True, xi=0.0, blocks=None):
    """SARA: an unweighted solve of (3) followed by n_reweight reweighted solves.
    Returns (x, list of per-round SDMMState)."""
    w = np.ones_like(psi.analysis(np.zeros((op.n, op.n))))
    st = sdmm(op, psi, y, eps, gamma, w, t_max, cg_iters, nu, None, xi, blocks)
    rounds = [st]
    alpha0 = psi.analysis(st.x)
    for k in range(1, n_reweight + 1):
        alpha = psi.analysis(st.x)
        delta = delta_schedule(alpha0, k, decay, delta0, delta_min)
        w = reweight(alpha, delta)
        x0 = st.x if warm_start else None
        st = sdmm(op, psi, y, eps, gamma, w, t_max, cg_iters, nu, x0, xi, blocks)
        rounds.append(st)
    return st.x, rounds
