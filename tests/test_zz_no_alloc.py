"""Allocation-free SARA analysis (purify_sara_fwd_static) against the oracle.

purify_sara_fwd_static serves callers that may not allocate device memory
once running (pipelines that reserve all memory up front, hosts that pass
only pre-sized buffers): its scratch is a fixed device array inside the
library.  Its output must equal the FP64 oracle's Psi^H x within the FP32
operator tolerance, on two calls in a row (the second reuses the scratch the
first left behind), up to the documented limit n = 512, and a repeat call
must not change the device's free memory.  The first call in a fresh process
(before any operator exists, so the library's device code is not loaded yet)
is checked in a child process.  This file sorts last so that a
stop-at-first-failure run has already run every other test.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import sara as osara
from paper_1406_0359_gb300 import synth
from tests._gpu import TOL, host, need_gpu, rel

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _call(L, x, c, n, levels):
    return L.purify_sara_fwd_static(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(c.data_ptr()), n, levels,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("n,levels", [(512, 4), (512, 1), (256, 4), (64, 3)])
def test_static_scratch_analysis_matches_oracle_twice(n, levels):
    need_gpu()
    from paper_1406_0359_gb300 import binding

    L = binding.lib()
    xs = [synth.random_image(n, seed) for seed in (1, 2)]
    xd = [torch.as_tensor(x, dtype=torch.float32, device="cuda") for x in xs]
    cd = [torch.full((9, n, n), float("nan"), dtype=torch.float32, device="cuda") for _ in xs]
    torch.cuda.synchronize()
    free = []
    for x, c in zip(xd, cd):  # two calls in a row share the fixed scratch
        rc = _call(L, x, c, n, levels)
        assert rc == 0, binding.purify_strerror(rc)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    assert free[1] == free[0]  # the repeat call reserved no device memory
    for x, c in zip(xs, cd):
        got = host(c)
        assert np.all(np.isfinite(got))
        assert rel(got, osara.analysis(x, levels)) < TOL["fp32"]


def test_static_scratch_rejects_oversize_request():
    need_gpu()
    from paper_1406_0359_gb300 import binding

    L = binding.lib()
    x = torch.zeros(1024, 1024, dtype=torch.float32, device="cuda")
    c = torch.zeros(9, 1024, 1024, dtype=torch.float32, device="cuda")
    assert _call(L, x, c, 1024, 4) == -1
    assert "512" in L.purify_last_error().decode()


_FRESH = r"""
import ctypes, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from oracle import sara as osara
from paper_1406_0359_gb300 import binding, synth
L = binding.lib()
n, levels = 128, 3
out = []
for seed in (3, 4):
    x = synth.random_image(n, seed)
    xd = torch.as_tensor(x, dtype=torch.float32, device="cuda")
    c = torch.empty((9, n, n), dtype=torch.float32, device="cuda")
    rc = L.purify_sara_fwd_static(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(c.data_ptr()), n, levels,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    ref = osara.analysis(x, levels)
    out.append(float(np.linalg.norm(c.cpu().numpy() - ref) / np.linalg.norm(ref)))
print(max(out))
"""


def test_static_scratch_first_call_in_a_fresh_process():
    """No operator has been created in the child, so the first call is the
    one that loads the device code and looks up the fixed array."""
    need_gpu()
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert float(r.stdout.strip().splitlines()[-1]) < TOL["fp32"]
