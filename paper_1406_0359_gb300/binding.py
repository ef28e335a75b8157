"""Thin ctypes binding of libpurify_gb300.so (C-ABI in include/purify.h).

Argument marshalling only: every step of the imaging path runs in the
library's CUDA kernels.  PyTorch supplies device memory and the current
stream.  The module-level functions carry the C entry points' names; the
``Operator`` class wraps one ``purify_op`` handle.

Raises ``RuntimeError`` when the library has not been built (there is no
fallback path).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpurify_gb300.so")

PURIFY_FP32, PURIFY_FP64 = 0, 1
_STATUS = {0: "ok", -1: "invalid argument", -2: "device allocation failed", -3: "CUDA runtime error",
           -4: "bounded device wait timed out", -5: "halting rule not met within t_max",
           -6: "device memory budget exceeded", -7: "request cancelled", -8: "solve produced non-finite values"}


class PurifyError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        super().__init__(f"{where}: {_STATUS.get(code, 'unknown')} ({code}) {detail}".rstrip())
        self.code = code


class purify_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("gamma", ctypes.c_double), ("nu", ctypes.c_double),
                ("t_max", ctypes.c_int), ("cg_iters", ctypes.c_int), ("xi", ctypes.c_double),
                ("n_reweight", ctypes.c_int), ("delta0", ctypes.c_double), ("delta_min", ctypes.c_double),
                ("delta_decay", ctypes.c_double), ("warm_start", ctypes.c_int), ("power_iters", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("gram", ctypes.c_int),
                ("eps_blocks", ctypes.POINTER(ctypes.c_double))]


class purify_op_options(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("chunk", ctypes.c_int)]


class purify_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("rounds", ctypes.c_int), ("converged", ctypes.c_int),
                ("objective", ctypes.c_double), ("residual", ctypes.c_double), ("nu", ctypes.c_double),
                ("gamma", ctypes.c_double), ("elapsed_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["purify_op_create", "purify_op_destroy", "purify_op_info", "purify_phi", "purify_phi_adj",
           "purify_sara_fwd", "purify_sara_adj", "purify_sdmm_solve", "purify_default_params",
           "purify_strerror", "purify_profile", "purify_profile_read", "purify_kernel_name",
           "purify_last_error", "purify_sara_fwd_static", "purify_gram", "purify_op_set_blocks",
           "purify_server_create", "purify_server_destroy", "purify_server_submit", "purify_server_step",
           "purify_server_result", "purify_estimate_bytes", "purify_op_create_ex", "purify_autotune",
           "purify_server_set_options", "purify_op_set_dictionary", "purify_op_dictionary",
           "purify_solve_begin", "purify_solve_step", "purify_solve_end", "purify_solve_state_bytes",
           "purify_solve_save", "purify_solve_load", "purify_set_wait_limit", "purify_wait_selftest",
           "purify_server_cancel", "purify_op_set_prior", "purify_batch_solve", "purify_server_set_batching",
           "purify_server_counts"]
KERNEL_KINDS = ["row_fwd", "col_fwd", "degrid", "grid", "gram", "col_inv", "row_inv", "sara_analysis",
                "sara_synthesis", "vector", "memset", "col_conv", "row_fwd_h", "row_inv_h", "tv"]

_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library (once).  Fails loudly if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1406_0359_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.purify_op_create.argtypes = [vp, i64, ci, ci, ci, ci, ci, vp, ctypes.POINTER(vp)]
    L.purify_op_destroy.argtypes = [vp]
    L.purify_op_info.argtypes = [vp] + [ctypes.POINTER(ci), ctypes.POINTER(i64), ctypes.POINTER(ci),
                                        ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci),
                                        ctypes.POINTER(i64)]
    for f in ("purify_phi", "purify_phi_adj", "purify_sara_fwd", "purify_sara_adj"):
        getattr(L, f).argtypes = [vp, vp, vp, vp]
    L.purify_sdmm_solve.argtypes = [vp, vp, ctypes.POINTER(purify_params), vp, ctypes.POINTER(purify_stats), vp]
    L.purify_default_params.argtypes = [ctypes.POINTER(purify_params)]
    L.purify_default_params.restype = None
    L.purify_strerror.argtypes = [ci]
    L.purify_strerror.restype = ctypes.c_char_p
    L.purify_profile.argtypes = [vp, ci]
    L.purify_profile_read.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    L.purify_kernel_name.argtypes = [ci]
    L.purify_kernel_name.restype = ctypes.c_char_p
    L.purify_sara_fwd_static.argtypes = [vp, vp, ci, ci, vp]
    L.purify_gram.argtypes = [vp, vp, vp, ci, vp]
    L.purify_op_set_blocks.argtypes = [vp, vp, ci, vp]
    L.purify_op_set_dictionary.argtypes = [vp, ctypes.c_uint]
    L.purify_op_dictionary.argtypes = [vp, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ci)]
    L.purify_server_create.argtypes = [i64, ci, ctypes.POINTER(vp)]
    L.purify_server_destroy.argtypes = [vp]
    L.purify_server_set_options.argtypes = [vp, ci, ctypes.POINTER(purify_op_options)]
    L.purify_server_submit.argtypes = [vp, vp, vp, i64, ci, ci, ci, ctypes.POINTER(purify_params),
                                       ctypes.POINTER(ci)]
    L.purify_server_step.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    L.purify_server_result.argtypes = [vp, ci, vp, ctypes.POINTER(purify_stats), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
    L.purify_estimate_bytes.argtypes = [i64, ci, ci, ci, ctypes.POINTER(i64)]
    L.purify_op_create_ex.argtypes = [vp, i64, ci, ci, ci, ci, ci, ctypes.POINTER(purify_op_options), vp,
                                      ctypes.POINTER(vp)]
    L.purify_autotune.argtypes = [vp, i64, ci, ci, ci, ci, vp, ctypes.POINTER(purify_op_options),
                                  ctypes.POINTER(ctypes.c_double)]
    L.purify_solve_begin.argtypes = [vp, vp, ctypes.POINTER(purify_params), vp]
    L.purify_solve_step.argtypes = [vp, ci, ctypes.POINTER(ci)]
    L.purify_solve_end.argtypes = [vp, vp, ctypes.POINTER(purify_stats), vp]
    L.purify_solve_state_bytes.argtypes = [vp, ctypes.POINTER(i64)]
    L.purify_solve_save.argtypes = [vp, vp, i64]
    L.purify_solve_load.argtypes = [vp, vp, i64]
    L.purify_set_wait_limit.argtypes = [ctypes.c_uint32]
    L.purify_wait_selftest.argtypes = [ci, vp]
    L.purify_server_cancel.argtypes = [vp, ci]
    L.purify_server_set_batching.argtypes = [vp, ci]
    L.purify_server_counts.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.purify_op_set_prior.argtypes = [vp, ci, ci]
    L.purify_batch_solve.argtypes = [ci, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(purify_params),
                                     ctypes.POINTER(vp), ctypes.POINTER(purify_stats), vp]
    L.purify_last_error.argtypes = []
    L.purify_last_error.restype = ctypes.c_char_p
    for f in EXPORTS:
        if f not in ("purify_default_params", "purify_strerror", "purify_kernel_name", "purify_last_error"):
            getattr(L, f).restype = ci
    _lib = L
    return L


def _check(rc: int, where: str, allow=()) -> int:
    if rc != 0 and rc not in allow:
        raise PurifyError(rc, where, lib().purify_last_error().decode(errors="replace"))
    return rc


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t: torch.Tensor, dtype: torch.dtype, shape=None) -> ctypes.c_void_p:
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous CUDA {dtype} tensor, got {t.dtype} on {t.device}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------- C entry points
def purify_op_create(uv: torch.Tensor, n: int, dwt_levels: int, precision: int = PURIFY_FP32,
                     oversample: int = 2, J: int = 8, stream=None) -> ctypes.c_void_p:
    """uv: CUDA float64 tensor (M, 2) in radians.  Returns the opaque handle."""
    h = ctypes.c_void_p()
    _check(lib().purify_op_create(_dptr(uv, torch.float64), uv.shape[0], n, oversample, J, dwt_levels,
                                  precision, _stream(stream), ctypes.byref(h)), "purify_op_create")
    return h


def purify_op_create_ex(uv: torch.Tensor, n: int, dwt_levels: int, precision: int = PURIFY_FP32, tile: int = 0,
                        chunk: int = 0, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    o = purify_op_options(tile, chunk)
    _check(lib().purify_op_create_ex(_dptr(uv, torch.float64), uv.shape[0], n, 2, 8, dwt_levels, precision,
                                     ctypes.byref(o), _stream(stream), ctypes.byref(h)), "purify_op_create_ex")
    return h


def purify_autotune(uv: torch.Tensor, n: int, dwt_levels: int, precision: int = PURIFY_FP32, reps: int = 3,
                    stream=None) -> tuple[int, int, float]:
    """(tile, chunk, ms per Phi + Phi^H) of the fastest work decomposition."""
    o = purify_op_options()
    ms = ctypes.c_double()
    _check(lib().purify_autotune(_dptr(uv, torch.float64), uv.shape[0], n, dwt_levels, precision, reps,
                                 _stream(stream), ctypes.byref(o), ctypes.byref(ms)), "purify_autotune")
    return o.tile, o.chunk, ms.value


def purify_op_destroy(h) -> None:
    if h:
        lib().purify_op_destroy(h)


def purify_op_info(h) -> dict:
    n, K, tile, ni, prec = (ctypes.c_int() for _ in range(5))
    M, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().purify_op_info(h, ctypes.byref(n), ctypes.byref(M), ctypes.byref(K), ctypes.byref(tile),
                                ctypes.byref(ni), ctypes.byref(prec), ctypes.byref(b)), "purify_op_info")
    return dict(n=n.value, M=M.value, K=K.value, tile=tile.value, n_items=ni.value, precision=prec.value,
                device_bytes=b.value)


def purify_phi(h, x_ptr, y_ptr, stream=None) -> None:
    _check(lib().purify_phi(h, x_ptr, y_ptr, _stream(stream)), "purify_phi")


def purify_phi_adj(h, y_ptr, x_ptr, stream=None) -> None:
    _check(lib().purify_phi_adj(h, y_ptr, x_ptr, _stream(stream)), "purify_phi_adj")


def purify_sara_fwd(h, x_ptr, c_ptr, stream=None) -> None:
    _check(lib().purify_sara_fwd(h, x_ptr, c_ptr, _stream(stream)), "purify_sara_fwd")


def purify_sara_adj(h, c_ptr, x_ptr, stream=None) -> None:
    _check(lib().purify_sara_adj(h, c_ptr, x_ptr, _stream(stream)), "purify_sara_adj")


def purify_sara_fwd_static(x_ptr, c_ptr, n: int, levels: int, stream=None) -> None:
    """Psi^H x without an operator and without device allocation (FP32,
    n <= 512; see include/purify.h)."""
    _check(lib().purify_sara_fwd_static(x_ptr, c_ptr, n, levels, _stream(stream)), "purify_sara_fwd_static")


def purify_op_set_blocks(h, block_ptr, R: int, stream=None) -> None:
    _check(lib().purify_op_set_blocks(h, block_ptr, R, _stream(stream)), "purify_op_set_blocks")


def purify_op_set_dictionary(h, mask: int) -> None:
    _check(lib().purify_op_set_dictionary(h, mask), "purify_op_set_dictionary")


def purify_op_dictionary(h) -> tuple[int, int]:
    """(mask, number of bases) of the operator's dictionary."""
    m, q = ctypes.c_uint(), ctypes.c_int()
    _check(lib().purify_op_dictionary(h, ctypes.byref(m), ctypes.byref(q)), "purify_op_dictionary")
    return m.value, q.value


def purify_gram(h, x_ptr, out_ptr, mode: int, stream=None) -> None:
    _check(lib().purify_gram(h, x_ptr, out_ptr, mode, _stream(stream)), "purify_gram")


def purify_default_params() -> purify_params:
    p = purify_params()
    lib().purify_default_params(ctypes.byref(p))
    return p


def purify_sdmm_solve(h, y_ptr, params: purify_params, x_ptr, stream=None) -> tuple[int, purify_stats]:
    st = purify_stats()
    rc = lib().purify_sdmm_solve(h, y_ptr, ctypes.byref(params), x_ptr, ctypes.byref(st), _stream(stream))
    _check(rc, "purify_sdmm_solve", allow=(-5,))
    return rc, st


def purify_solve_begin(h, y_ptr, params: purify_params, stream=None) -> None:
    _check(lib().purify_solve_begin(h, y_ptr, ctypes.byref(params), _stream(stream)), "purify_solve_begin")


def purify_solve_step(h, max_iters: int) -> bool:
    """Run up to max_iters SDMM iterations; True once the solve has finished."""
    done = ctypes.c_int()
    _check(lib().purify_solve_step(h, max_iters, ctypes.byref(done)), "purify_solve_step")
    return bool(done.value)


def purify_solve_end(h, x_ptr, stream=None) -> tuple[int, purify_stats]:
    st = purify_stats()
    rc = lib().purify_solve_end(h, x_ptr, ctypes.byref(st), _stream(stream))
    _check(rc, "purify_solve_end", allow=(-5,))
    return rc, st


def purify_solve_state_bytes(h) -> int:
    b = ctypes.c_int64()
    _check(lib().purify_solve_state_bytes(h, ctypes.byref(b)), "purify_solve_state_bytes")
    return b.value


def purify_solve_save(h) -> bytes:
    buf = ctypes.create_string_buffer(purify_solve_state_bytes(h))
    _check(lib().purify_solve_save(h, buf, len(buf)), "purify_solve_save")
    return buf.raw


def purify_solve_load(h, state: bytes) -> None:
    buf = ctypes.create_string_buffer(state, len(state))
    _check(lib().purify_solve_load(h, buf, len(state)), "purify_solve_load")


def purify_set_wait_limit(spins: int) -> None:
    _check(lib().purify_set_wait_limit(spins), "purify_set_wait_limit")


def purify_wait_selftest(deliver: bool, stream=None) -> int:
    """Status of the bounded-wait self-test (0, or -4 when the wait gave up)."""
    return lib().purify_wait_selftest(int(deliver), _stream(stream))


def purify_strerror(code: int) -> str:
    return lib().purify_strerror(code).decode()


def purify_profile(h, enable: bool) -> None:
    _check(lib().purify_profile(h, int(enable)), "purify_profile")


def purify_profile_read(h, kind: int) -> tuple[float, int]:
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(lib().purify_profile_read(h, kind, ctypes.byref(ms), ctypes.byref(n)), "purify_profile_read")
    return ms.value, n.value


def purify_kernel_name(kind: int) -> str:
    return lib().purify_kernel_name(kind).decode()


# ------------------------------------------------------------- convenience
@dataclass
class SolveResult:
    x: torch.Tensor
    stats: dict
    status: int


class Operator:
    """One measurement operator + SARA dictionary on the current CUDA device."""

    def __init__(self, uv, n: int, levels: int, precision: str = "fp32", stream=None, tile: int = 0,
                 chunk: int = 0):
        self.n, self.levels = n, levels
        self.prec = PURIFY_FP32 if precision == "fp32" else PURIFY_FP64
        self.rdtype = torch.float32 if self.prec == PURIFY_FP32 else torch.float64
        self.cdtype = torch.complex64 if self.prec == PURIFY_FP32 else torch.complex128
        uv_t = torch.as_tensor(uv, dtype=torch.float64)
        if not uv_t.is_cuda:
            uv_t = uv_t.cuda()
        self.M = uv_t.shape[0]
        if tile or chunk:
            self.h = purify_op_create_ex(uv_t.contiguous(), n, levels, self.prec, tile, chunk, stream=stream)
        else:
            self.h = purify_op_create(uv_t.contiguous(), n, levels, self.prec, stream=stream)

    def close(self) -> None:
        if getattr(self, "h", None):
            purify_op_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return purify_op_info(self.h)

    def profile(self, enable: bool) -> None:
        purify_profile(self.h, enable)

    def kernel_times(self) -> dict:
        """{kind: (total_ms, launches)} accumulated since profiling was enabled."""
        return {KERNEL_KINDS[k]: purify_profile_read(self.h, k) for k in range(len(KERNEL_KINDS))}

    def phi(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        n = self.n
        y = out if out is not None else torch.empty(self.M, dtype=self.cdtype, device=x.device)
        purify_phi(self.h, _dptr(x, self.rdtype, (n, n)), _dptr(y, self.cdtype, (self.M,)), stream)
        return y

    def phi_adj(self, y: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        n = self.n
        x = out if out is not None else torch.empty(n, n, dtype=self.rdtype, device=y.device)
        purify_phi_adj(self.h, _dptr(y, self.cdtype, (self.M,)), _dptr(x, self.rdtype, (n, n)), stream)
        return x

    def set_blocks(self, block_ids, R: int, stream=None) -> None:
        """Split the visibilities into R blocks (caller-order int32 ids in [0, R))."""
        b = torch.as_tensor(block_ids, dtype=torch.int32).cuda().contiguous()
        purify_op_set_blocks(self.h, _dptr(b, torch.int32, (self.M,)), R, stream)
        self.R = R

    def gram(self, x: torch.Tensor, mode: int = 1, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Re(Phi^H Phi x); mode 0 NUFFT, 1 precomputed PSF convolution."""
        n = self.n
        o = out if out is not None else torch.empty(n, n, dtype=self.rdtype, device=x.device)
        purify_gram(self.h, _dptr(x, self.rdtype, (n, n)), _dptr(o, self.rdtype, (n, n)), mode, stream)
        return o

    def set_dictionary(self, mask: int) -> None:
        """Bases of Psi: bit 0 Dirac, bit K DbK (default 0x1FF, SARA)."""
        purify_op_set_dictionary(self.h, mask)

    def set_prior(self, prior: str = "l1", tv_iters: int = 20) -> None:
        """First SDMM block: "l1" (analysis over the dictionary) or "tv"."""
        _check(lib().purify_op_set_prior(self.h, {"l1": 0, "tv": 1}[prior], tv_iters), "purify_op_set_prior")

    def dictionary(self) -> tuple[int, int]:
        """(mask, number of bases q) of Psi."""
        return purify_op_dictionary(self.h)

    def sara_fwd(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        n, q = self.n, self.dictionary()[1]
        c = out if out is not None else torch.empty(q, n, n, dtype=self.rdtype, device=x.device)
        purify_sara_fwd(self.h, _dptr(x, self.rdtype, (n, n)), _dptr(c, self.rdtype, (q, n, n)), stream)
        return c

    def sara_adj(self, c: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        n, q = self.n, self.dictionary()[1]
        x = out if out is not None else torch.empty(n, n, dtype=self.rdtype, device=c.device)
        purify_sara_adj(self.h, _dptr(c, self.rdtype, (q, n, n)), _dptr(x, self.rdtype, (n, n)), stream)
        return x

    @staticmethod
    def params(eps: float, t_max: int = 200, cg_iters: int = 10, n_reweight: int = 0, gamma: float = 0.0,
               nu: float = 0.0, xi: float = 0.0, delta0: float = 0.0, delta_min: float = 0.0,
               delta_decay: float = 0.1, warm_start: bool = True, power_iters: int = 30, use_graph: bool = True,
               gram: int = -1) -> purify_params:
        p = purify_default_params()
        p.eps, p.gamma, p.nu, p.t_max, p.cg_iters = eps, gamma, nu, t_max, cg_iters
        p.xi, p.n_reweight, p.delta0, p.delta_min = xi, n_reweight, delta0, delta_min
        p.delta_decay, p.warm_start, p.power_iters, p.use_graph = delta_decay, int(warm_start), power_iters, int(use_graph)
        p.gram = gram
        return p

    def solve_begin(self, y: torch.Tensor, eps: float, stream=None, **kw) -> None:
        """Start a resumable solve (purify_solve_begin); keyword arguments as solve()."""
        self._y_keep = y
        purify_solve_begin(self.h, _dptr(y, self.cdtype, (self.M,)), self.params(eps, **kw), stream)

    def solve_step(self, max_iters: int) -> bool:
        return purify_solve_step(self.h, max_iters)

    def solve_end(self, out: torch.Tensor | None = None, stream=None) -> SolveResult:
        n = self.n
        x = out if out is not None else torch.empty(n, n, dtype=self.rdtype, device="cuda")
        rc, st = purify_solve_end(self.h, _dptr(x, self.rdtype, (n, n)), stream)
        return SolveResult(x, st.as_dict(), rc)

    def save_state(self) -> bytes:
        return purify_solve_save(self.h)

    def load_state(self, state: bytes) -> None:
        purify_solve_load(self.h, state)

    def solve(self, y: torch.Tensor, eps: float, t_max: int = 200, cg_iters: int = 10, n_reweight: int = 0,
              gamma: float = 0.0, nu: float = 0.0, xi: float = 0.0, delta0: float = 0.0,
              delta_min: float = 0.0, delta_decay: float = 0.1, warm_start: bool = True,
              power_iters: int = 30, use_graph: bool = True, gram: int = -1, eps_blocks=None,
              out: torch.Tensor | None = None, stream=None) -> SolveResult:
        p = purify_default_params()
        p.eps, p.gamma, p.nu, p.t_max, p.cg_iters = eps, gamma, nu, t_max, cg_iters
        p.xi, p.n_reweight, p.delta0, p.delta_min = xi, n_reweight, delta0, delta_min
        p.delta_decay, p.warm_start, p.power_iters, p.use_graph = delta_decay, int(warm_start), power_iters, int(use_graph)
        p.gram = gram
        if eps_blocks is not None:
            arr = (ctypes.c_double * len(eps_blocks))(*[float(e) for e in eps_blocks])
            p.eps_blocks = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
            self._eps_keep = arr
        n = self.n
        x = out if out is not None else torch.empty(n, n, dtype=self.rdtype, device=y.device)
        rc, st = purify_sdmm_solve(self.h, _dptr(y, self.cdtype, (self.M,)), p, _dptr(x, self.rdtype, (n, n)),
                                   stream)
        return SolveResult(x, st.as_dict(), rc)


def batch_solve(ops: list, ys: list, eps: list, stream=None, **kw) -> list:
    """purify_batch_solve over Operators `ops` with visibilities `ys` and
    per-instance bounds `eps`; keyword arguments (shared, or a list per
    instance for gamma / nu) as Operator.solve.  Returns SolveResults."""
    count = len(ops)
    per = {k: kw.pop(k) for k in ("gamma", "nu") if isinstance(kw.get(k), (list, tuple))}
    P = (purify_params * count)()
    st = (purify_stats * count)()
    xs = [torch.empty(o.n, o.n, dtype=o.rdtype, device="cuda") for o in ops]
    for i, o in enumerate(ops):
        extra = {k: v[i] for k, v in per.items()}
        P[i] = Operator.params(float(eps[i]), **kw, **extra)
    H = (ctypes.c_void_p * count)(*[o.h for o in ops])
    Y = (ctypes.c_void_p * count)(*[_dptr(y, o.cdtype, (o.M,)).value for y, o in zip(ys, ops)])
    X = (ctypes.c_void_p * count)(*[x.data_ptr() for x in xs])
    rc = lib().purify_batch_solve(count, H, Y, P, X, st, _stream(stream))
    _check(rc, "purify_batch_solve", allow=(-5,))
    return [SolveResult(x, s.as_dict(), rc) for x, s in zip(xs, st)]


def purify_estimate_bytes(M: int, n: int, levels: int, precision: int = PURIFY_FP32) -> int:
    b = ctypes.c_int64()
    _check(lib().purify_estimate_bytes(M, n, levels, precision, ctypes.byref(b)), "purify_estimate_bytes")
    return b.value


class Server:
    """Continuous-batching request server (C-ABI purify_server_*).  Requests
    are host arrays; results come back as host arrays."""

    def __init__(self, budget_bytes: int, max_slots: int):
        self.h = ctypes.c_void_p()
        _check(lib().purify_server_create(int(budget_bytes), int(max_slots), ctypes.byref(self.h)),
               "purify_server_create")
        self.meta = {}

    def close(self) -> None:
        if self.h:
            lib().purify_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, uv, y, n: int, levels: int, eps: float, precision: str = "fp32", **kw) -> int:
        import numpy as np

        prec = PURIFY_FP32 if precision == "fp32" else PURIFY_FP64
        uv = np.ascontiguousarray(uv, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.complex64 if prec == PURIFY_FP32 else np.complex128)
        p = purify_default_params()
        p.eps = eps
        for k, v in kw.items():
            setattr(p, k, v)
        rid = ctypes.c_int()
        _check(lib().purify_server_submit(self.h, uv.ctypes.data_as(ctypes.c_void_p),
                                          y.ctypes.data_as(ctypes.c_void_p), uv.shape[0], n, levels, prec,
                                          ctypes.byref(p), ctypes.byref(rid)), "purify_server_submit")
        self.meta[rid.value] = (n, prec)
        return rid.value

    def set_options(self, n: int, tile: int, chunk: int) -> None:
        o = purify_op_options(tile, chunk)
        _check(lib().purify_server_set_options(self.h, n, ctypes.byref(o)), "purify_server_set_options")

    def set_batching(self, enable: bool) -> None:
        _check(lib().purify_server_set_batching(self.h, int(enable)), "purify_server_set_batching")

    def counts(self) -> tuple[int, int]:
        """(solve-iterations launched in batched groups, on their own)."""
        b, s = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().purify_server_counts(self.h, ctypes.byref(b), ctypes.byref(s)), "purify_server_counts")
        return b.value, s.value

    def cancel(self, rid: int) -> None:
        _check(lib().purify_server_cancel(self.h, rid), "purify_server_cancel")

    def step(self) -> tuple[int, int]:
        a, q = ctypes.c_int(), ctypes.c_int()
        _check(lib().purify_server_step(self.h, ctypes.byref(a), ctypes.byref(q)), "purify_server_step")
        return a.value, q.value

    def result(self, rid: int):
        """None while pending, else (image, stats, latency_s, queue_s)."""
        import numpy as np

        n, prec = self.meta[rid]
        x = np.empty((n, n), dtype=np.float32 if prec == PURIFY_FP32 else np.float64)
        st = purify_stats()
        lat, qs = ctypes.c_double(), ctypes.c_double()
        rc = lib().purify_server_result(self.h, rid, x.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st),
                                        ctypes.byref(lat), ctypes.byref(qs))
        if rc == 0:
            return None
        _check(rc if rc < 0 else 0, "purify_server_result")
        return x, st.as_dict(), lat.value, qs.value


def solve_from_host(uv_host, y_host, n: int, levels: int, eps: float, precision: str = "fp32",
                    **kw) -> SolveResult:
    """End-to-end call on host arrays: copy uv and y to the device, build the
    operator, solve, and copy the image back to host memory."""
    dev = torch.device("cuda")
    uv = torch.as_tensor(uv_host, dtype=torch.float64).to(dev, non_blocking=True)
    op = Operator(uv, n, levels, precision)
    y = torch.as_tensor(y_host).to(dev, dtype=op.cdtype, non_blocking=True)
    res = op.solve(y, eps, **kw)
    x_host = res.x.cpu()
    op.close()
    return SolveResult(x_host, res.stats, res.status)
