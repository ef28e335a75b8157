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
