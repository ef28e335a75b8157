"""Shared set-up for the GPU parity tests: build the library once, make
seeded problems, compare with the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import simulate
from oracle.nufft import NUFFT
from paper_1406_0359_gb300 import synth

TOL = {"fp32": 1e-5, "fp64": 1e-11}  # per-operator relative L2 error bound


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_0359_gb300 import build

    build.build()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(a, prec):
    dt = {"fp32": torch.float32, "fp64": torch.float64}[prec]
    ct = {"fp32": torch.complex64, "fp64": torch.complex128}[prec]
    a = np.asarray(a)
    if np.iscomplexobj(a):
        return torch.as_tensor(a).to("cuda", ct).contiguous()
    return torch.as_tensor(a).to("cuda", dt).contiguous()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def measured_problem(n, M, seed, n_blobs=3, n_points=10, isnr=30.0):
    """Seeded sky, coverage and noisy visibilities (y from the oracle's Phi)."""
    uv = synth.uv_coverage(M, n, seed)
    x_true = synth.sky(n, seed, n_blobs, n_points)
    op = NUFFT(uv, n)
    a, b = synth.noise_draws(M, seed)
    y, sigma = simulate.add_noise(op.phi(x_true), isnr, a, b)
    eps = simulate.epsilon(sigma, M)
    return dict(uv=uv, x_true=x_true, op=op, y=y, eps=eps, sigma=sigma, n=n, M=M)
