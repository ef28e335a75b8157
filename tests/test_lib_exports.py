"""The C-ABI library builds for sm_103a and exports every entry point that
include/purify.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(purify_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_every_declared_symbol():
    from paper_1406_0359_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1406_0359_gb300 import binding

    assert set(binding.EXPORTS) == set(names)


def test_strerror_without_gpu():
    from paper_1406_0359_gb300 import binding, build

    build.build()
    assert binding.purify_strerror(0) == "ok"
    assert "invalid" in binding.purify_strerror(-1)
    p = binding.purify_default_params()
    assert p.t_max == 200 and p.cg_iters == 10 and p.use_graph == 1


def test_memory_estimate_is_monotone_without_gpu():
    from paper_1406_0359_gb300 import binding, build

    build.build()
    a = binding.purify_estimate_bytes(100_000, 256, 4)
    assert binding.purify_estimate_bytes(200_000, 256, 4) > a
    assert binding.purify_estimate_bytes(100_000, 512, 4) > a
    assert binding.purify_estimate_bytes(100_000, 256, 4, binding.PURIFY_FP64) > a


def test_invalid_arguments_are_rejected_before_any_device_work():
    """Argument checks of the C-ABI run before any CUDA call, so they can be
    exercised without a GPU: every bad size, option or null pointer returns
    PURIFY_ERR_INVALID (the uv pointer below is never dereferenced)."""
    from paper_1406_0359_gb300 import binding, build

    build.build()
    L = binding.lib()
    INV = -1  # PURIFY_ERR_INVALID
    fake = ctypes.c_void_p(256)
    h = ctypes.c_void_p()
    F32 = binding.PURIFY_FP32

    def create(uv=fake, M=4096, n=64, over=2, J=8, levels=3, prec=F32, out=True):
        return L.purify_op_create(uv, M, n, over, J, levels, prec, None, ctypes.byref(h) if out else None)

    bad = [dict(uv=None), dict(M=0), dict(M=1 << 31), dict(n=8), dict(n=100), dict(n=4096), dict(over=3),
           dict(J=6), dict(levels=0), dict(n=16, levels=4), dict(prec=7), dict(out=False)]
    for kw in bad:
        assert create(**kw) == INV, kw
    assert h.value is None
    opt = binding.purify_op_options(tile=12, chunk=0)
    assert L.purify_op_create_ex(fake, 4096, 64, 2, 8, 3, F32, ctypes.byref(opt), None, ctypes.byref(h)) == INV
    opt = binding.purify_op_options(tile=8, chunk=32)
    assert L.purify_op_create_ex(fake, 4096, 64, 2, 8, 3, F32, ctypes.byref(opt), None, ctypes.byref(h)) == INV
    for f in ("purify_phi", "purify_phi_adj", "purify_sara_fwd", "purify_sara_adj"):
        assert getattr(L, f)(None, fake, fake, None) == INV, f
    assert L.purify_gram(None, fake, fake, 1, None) == INV
    assert L.purify_op_set_dictionary(None, 1) == INV
    assert L.purify_op_destroy(None) == 0


def test_resume_and_diagnostic_calls_reject_bad_arguments_without_gpu():
    from paper_1406_0359_gb300 import binding, build

    build.build()
    L = binding.lib()
    fake = ctypes.c_void_p(256)
    done = ctypes.c_int()
    b = ctypes.c_int64()
    p = binding.purify_default_params()
    assert L.purify_solve_begin(None, fake, ctypes.byref(p), None) == -1
    assert L.purify_solve_begin(fake, None, ctypes.byref(p), None) == -1
    assert L.purify_solve_step(None, 1, ctypes.byref(done)) == -1
    assert L.purify_solve_end(None, fake, None, None) == -1
    assert L.purify_solve_state_bytes(None, ctypes.byref(b)) == -1
    assert L.purify_solve_save(None, fake, 16) == -1
    assert L.purify_solve_load(None, fake, 16) == -1
    assert L.purify_server_cancel(None, 1) == -1
    assert binding.purify_strerror(-7) == "request cancelled"
    assert "non-finite" in binding.purify_strerror(-8)
