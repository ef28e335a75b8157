"""Dense tiny-problem helpers for oracle pins (n = 8): Phi and Psi^H as explicit
matrices built column by column from the oracle's own operators."""
import math

import numpy as np

from oracle import sara, simulate
from oracle import sdmm as S
from oracle.nufft import NUFFT
from paper_1406_0359_gb300 import synth


class DenseOp:
    def __init__(self, Phi, n):
        self.Phi, self.n, self.M = Phi, n, Phi.shape[0]

    def phi(self, x):
        return self.Phi @ np.asarray(x).reshape(-1)

    def phi_adj_real(self, y):
        return (self.Phi.conj().T @ y).real.reshape(self.n, self.n)

    def gram_real(self, x):
        return self.phi_adj_real(self.phi(x))


class DensePsi:
    def __init__(self, Psih, n):
        self.Psih, self.n = Psih, n

    def analysis(self, x):
        return self.Psih @ np.asarray(x).reshape(-1)

    def synthesis(self, c):
        return (self.Psih.T @ c).reshape(self.n, self.n)


def tiny_problem(n=8, M=96, levels=1, seed=11, bases=sara.ALL_BASES):
    uv = synth.uv_coverage(M, n, seed)
    op = NUFFT(uv, n)
    N = n * n
    eye = np.eye(N)
    Phi = np.stack([op.phi(e.reshape(n, n)) for e in eye], axis=1)
    Psih = np.stack([sara.analysis(e.reshape(n, n), levels, bases).ravel() for e in eye], axis=1)
    dop, dpsi = DenseOp(Phi, n), DensePsi(Psih, n)
    x_true = synth.sky(n, seed, 1, 3)
    y0 = dop.phi(x_true)
    a, b = synth.noise_draws(M, seed)
    y, sig = simulate.add_noise(y0, 30.0, a, b)
    eps = simulate.epsilon(sig, M)
    nu = 1.0 / math.sqrt(S.operator_norm_sq(dop, 100))
    return dict(op=op, dop=dop, dpsi=dpsi, Phi=Phi, Psih=Psih, y=y, eps=eps, nu=nu,
                x_true=x_true, n=n, M=M, levels=levels)
