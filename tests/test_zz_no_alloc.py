"""Allocation-free SARA analysis (purify_sara_fwd_static) against the operator path.

purify_sara_fwd_static serves callers that may not allocate device memory
once running (pipelines that reserve all memory up front, hosts that pass
only pre-sized buffers): its scratch is a fixed device array inside the
library.  Its output must equal purify_sara_fwd's within the FP32 operator
tolerance, on two calls in a row (the second reuses the scratch the first
left behind).  This file sorts last so that a stop-at-first-failure run has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1406_0359_gb300 import synth
from tests._gpu import TOL, host, need_gpu, rel

pytestmark = pytest.mark.gpu


def test_static_scratch_analysis_matches_operator_twice():
    need_gpu()
    from paper_1406_0359_gb300 import binding

    L = binding.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, levels in ((256, 4), (64, 3)):
        op = binding.Operator(torch.as_tensor(synth.uv_coverage(64, n, 1)).cuda(), n, levels, "fp32")
        for seed in (1, 2):  # two calls in a row share the fixed scratch
            x = torch.as_tensor(synth.random_image(n, seed), dtype=torch.float32, device="cuda")
            ref = host(op.sara_fwd(x))
            c = torch.full((9, n, n), float("nan"), dtype=torch.float32, device="cuda")
            rc = L.purify_sara_fwd_static(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(c.data_ptr()), n, levels,
                                          stream)
            assert rc == 0, binding.purify_strerror(rc)
            got = host(c)
            assert np.all(np.isfinite(got))
            assert rel(got, ref) < TOL["fp32"]
        op.close()


def test_static_scratch_rejects_oversize_request():
    need_gpu()
    from paper_1406_0359_gb300 import binding

    L = binding.lib()
    x = torch.zeros(1024, 1024, dtype=torch.float32, device="cuda")
    c = torch.zeros(9, 1024, 1024, dtype=torch.float32, device="cuda")
    rc = L.purify_sara_fwd_static(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(c.data_ptr()), 1024, 4,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert "512" in L.purify_last_error().decode()
