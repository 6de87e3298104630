"""Thin ctypes binding of the C ABI in include/wd.h (argument marshalling only).

Every numerical step runs in the CUDA library ``libwdcg.so``; this module only converts torch
tensors to pointers and status codes to exceptions. Importing it fails loudly if the library has
not been built (``python -m paper_2111_14958_gb300.build``): there is no CPU fallback.

Low-level functions carry the C names (``wd_create``, ``wd_load_gauge``, ``wd_apply``,
``cg_solve``, ...); :class:`WilsonDirac` wraps them for torch users.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwdcg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python -m paper_2111_14958_gb300.build); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

# status codes (include/wd.h)
WD_OK = 0
WD_NOT_CONVERGED = 1
WD_EINVAL = -1
WD_ENOMEM = -2
WD_ECUDA = -3
WD_ENOTUNITARY = -4
WD_BREAKDOWN = -5
WD_ENOGAUGE = -6
STATUS_NAMES = {0: "WD_OK", 1: "WD_NOT_CONVERGED", -1: "WD_EINVAL", -2: "WD_ENOMEM", -3: "WD_ECUDA",
                -4: "WD_ENOTUNITARY", -5: "WD_BREAKDOWN", -6: "WD_ENOGAUGE"}

WD_PREC_F64 = 64
WD_PREC_F32 = 32
WD_PREC_MIXED_F32 = 6432
WD_PREC_MIXED_F16 = 6416
WD_EVEN_ODD = 0x10000

WD_OPT_RELIABLE_DELTA = 1
WD_OPT_USE_GRAPH = 2
WD_OPT_BLOCK_DSLASH = 3
WD_OPT_BLOCK_BLAS = 4
WD_OPT_MAX_RESTARTS = 5


WD_OPT_MULTI_GROUP = 6
WD_OPT_MULTI_SITES = 7
WD_OPT_DF_UPDATES = 8
WD_OPT_APPLY_DF = 9
WD_OPT_CG_FORM = 10
WD_OPT_DSLASH_VARIANT = 11
WD_OPT_LOOP_WAIT_LIMIT = 12
WD_OPT_RESIDUAL_HISTORY = 13
WD_OPT_APPLY_INNER = 14
WD_OPT_MULTI_RHS_PER_THREAD = 15
WD_OPT_DSLASH_TMA = 16
WD_OPT_DSLASH_SCHEDULE = 17
WD_OPT_LOOP_TIME_BASIS = 18


class WdMultiStats(ctypes.Structure):
    _fields_ = [("nrhs", ctypes.c_int), ("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("reliable_updates", ctypes.c_int), ("group", ctypes.c_int), ("sites_per_block", ctypes.c_int),
                ("status", ctypes.c_int), ("rhs_per_thread", ctypes.c_int), ("solve_ms", ctypes.c_double),
                ("dslash_ms", ctypes.c_double)]


class WdRequest(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("kappa", ctypes.c_double), ("eps", ctypes.c_double),
                ("gauge_seed", ctypes.c_ulonglong), ("source_seed", ctypes.c_ulonglong),
                ("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("precision", ctypes.c_int),
                ("boundary_set", ctypes.c_int), ("boundary", ctypes.c_int * 4),
                ("src_host", ctypes.c_void_p), ("x_host", ctypes.c_void_p)]


class WdResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int),
                ("slot", ctypes.c_int), ("true_rel_residual", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("batch", ctypes.c_int)]


class WdServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("admitted", ctypes.c_longlong),
                ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("warm_hits", ctypes.c_longlong), ("evictions", ctypes.c_longlong), ("pending", ctypes.c_int),
                ("used_bytes", ctypes.c_double), ("peak_bytes", ctypes.c_double),
                ("batches", ctypes.c_longlong), ("batched_requests", ctypes.c_longlong)]


class WdStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("reliable_updates", ctypes.c_int), ("dslash_calls", ctypes.c_int),
                ("dslash_calls_f64", ctypes.c_int), ("status", ctypes.c_int),
                ("loop_mode", ctypes.c_int), ("loop_lanes", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("loop_ms", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_sig = {
    "wd_create": (_I, [ctypes.POINTER(_I), _D, ctypes.POINTER(_I), _I, _P, ctypes.POINTER(_P)]),
    "wd_destroy": (None, [_P]),
    "wd_set_kappa": (_I, [_P, _D]),
    "wd_load_gauge": (_I, [_P, _P, _I, _I, ctypes.POINTER(_D)]),
    "wd_apply": (_I, [_P, _P, _P, _I]),
    "cg_solve": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "cg_solve_batch": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_D), _I,
                            ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "wd_cg_state_size": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "wd_cg_save_state": (_I, [_P, _P, ctypes.c_size_t]),
    "cg_resume": (_I, [_P, _P, ctypes.c_size_t, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "wd_set_option": (_I, [_P, _I, _D]),
    "wd_get_stats": (_I, [_P, ctypes.POINTER(WdStats)]),
    "wd_get_residual_history": (_I, [_P, ctypes.POINTER(_D), _I, ctypes.POINTER(_I)]),
    "wd_time_dslash": (_I, [_P, _I, _I, ctypes.POINTER(_D)]),
    "wd_apply_multi": (_I, [_P, _P, _P, _I, _I]),
    "cg_solve_multi": (_I, [_P, _P, _P, _I, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "wd_get_multi_stats": (_I, [_P, ctypes.POINTER(WdMultiStats)]),
    "wd_generate_gauge": (_I, [_P, _D, ctypes.c_ulonglong, _I, _P]),
    "wd_generate_source": (_I, [_P, ctypes.c_ulonglong, _P]),
    "wd_coo_build": (_I, [_P, _P, _P, _P, _P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    "wd_coo_spmv": (_I, [_P, ctypes.c_longlong, _P, _P, _P, _P, _P]),
    "wd_dslash_noalloc": (_I, [ctypes.POINTER(_I), _D, ctypes.POINTER(_I), _P, _P, _P, _I, _P, _P]),
    "wd_measure_fp64_peak": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "wd_server_create": (_I, [_D, _I, ctypes.POINTER(_P)]),
    "wd_server_submit": (_I, [_P, ctypes.POINTER(WdRequest), ctypes.POINTER(ctypes.c_longlong)]),
    "wd_server_wait": (_I, [_P, ctypes.c_longlong, ctypes.POINTER(WdResult)]),
    "wd_server_poll": (_I, [_P, ctypes.c_longlong, ctypes.POINTER(WdResult), ctypes.POINTER(_I)]),
    "wd_server_get_stats": (_I, [_P, ctypes.POINTER(WdServerStats)]),
    "wd_server_set_max_batch": (_I, [_P, _I]),
    "wd_server_set_policy": (_I, [_P, _I, _D]),
    "wd_server_destroy": (None, [_P]),
    "wd_last_error": (ctypes.c_char_p, []),
    "wd_version": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class WdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.wd_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def _check(status: int, where: str, allow=(WD_OK,)) -> int:
    if status not in allow:
        raise WdError(status, where)
    return status


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream_handle(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ------------------------------------------------------------------ C-named functions

def wd_version() -> str:
    return _lib.wd_version().decode()


def wd_last_error() -> str:
    return _lib.wd_last_error().decode(errors="replace")


def wd_create(dims, kappa: float, boundary=(1, 1, 1, -1), precision: int = WD_PREC_F64, stream=None):
    """Create a context; returns an opaque handle (int). Raises WdError on failure."""
    d = (_I * 4)(*[int(v) for v in dims])
    b = (_I * 4)(*[int(v) for v in boundary]) if boundary is not None else None
    out = _P()
    _check(_lib.wd_create(d, float(kappa), b, int(precision), _P(_stream_handle(stream)), ctypes.byref(out)),
           "wd_create")
    return out.value


def wd_set_kappa(ctx, kappa: float) -> None:
    _check(_lib.wd_set_kappa(_P(ctx), float(kappa)), "wd_set_kappa")


def wd_destroy(ctx) -> None:
    _lib.wd_destroy(_P(ctx))


def wd_load_gauge(ctx, U: torch.Tensor, compress12: bool = False, check: bool = True) -> float:
    """Load links (complex128 [Lt,Lz,Ly,Lx,4,3,3], host or device). Returns the max SU(3) deviation."""
    if U.dtype != torch.complex128 or not U.is_contiguous():
        raise ValueError("U must be a contiguous complex128 tensor")
    dev = _D(0.0)
    st = _lib.wd_load_gauge(_P(ctx), _P(_ptr(U)), int(U.is_cuda), int(compress12), ctypes.byref(dev))
    _check(st, "wd_load_gauge", allow=(WD_OK,) if check else (WD_OK, WD_ENOTUNITARY))
    return dev.value


def wd_apply(ctx, inp: torch.Tensor, out: torch.Tensor, dagger: bool = False) -> None:
    """inp and out: contiguous CUDA tensors of one complex dtype and size (complex64 for FP32
    contexts, complex128 otherwise; the library checks the context side)."""
    if (inp.dtype not in (torch.complex64, torch.complex128) or out.dtype != inp.dtype or
            out.numel() != inp.numel() or not (inp.is_cuda and out.is_cuda) or
            not (inp.is_contiguous() and out.is_contiguous())):
        raise ValueError("wd_apply: in and out must be contiguous CUDA tensors of one complex dtype and size")
    _check(_lib.wd_apply(_P(ctx), _P(_ptr(inp)), _P(_ptr(out)), int(bool(dagger))), "wd_apply")


def cg_solve(ctx, src: torch.Tensor, x: torch.Tensor, tol: float, maxit: int):
    """Returns (status, iterations, true relative residual); x is updated in place. src and x are
    contiguous complex128 CUDA tensors of one size, for every precision."""
    for t in (src, x):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("cg_solve: src and x must be contiguous complex128 CUDA tensors")
    if src.numel() != x.numel():
        raise ValueError("cg_solve: src and x must have the same size")
    it = _I(0)
    res = _D(0.0)
    st = _lib.cg_solve(_P(ctx), _P(_ptr(src)), _P(_ptr(x)), float(tol), int(maxit), ctypes.byref(it),
                       ctypes.byref(res))
    _check(st, "cg_solve", allow=(WD_OK, WD_NOT_CONVERGED, WD_BREAKDOWN))
    return st, it.value, res.value


def cg_solve_batch(ctxs, srcs, xs, tols, maxit: int):
    """n independent solves, each bitwise as cg_solve alone (one loop launch per pass where they share
    a shape). Returns (status, iterations, true relative residuals, per-problem statuses); the x
    tensors are updated in place."""
    n = len(ctxs)
    if not (len(srcs) == len(xs) == len(tols) == n):
        raise ValueError("ctxs, srcs, xs and tols must have the same length")
    for t in list(srcs) + list(xs):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("sources and solutions must be contiguous complex128 CUDA tensors")
    c = (_P * n)(*[_P(v) for v in ctxs])
    sp = (_P * n)(*[_P(_ptr(t)) for t in srcs])
    xp = (_P * n)(*[_P(_ptr(t)) for t in xs])
    tl = (_D * n)(*[float(t) for t in tols])
    it, res, sts = (_I * n)(), (_D * n)(), (_I * n)()
    st = _lib.cg_solve_batch(c, n, sp, xp, tl, int(maxit), it, res, sts)
    _check(st, "cg_solve_batch", allow=(WD_OK, WD_NOT_CONVERGED, WD_BREAKDOWN))
    return st, list(it), list(res), list(sts)


def wd_cg_state_size(ctx) -> int:
    n = ctypes.c_size_t()
    _check(_lib.wd_cg_state_size(_P(ctx), ctypes.byref(n)), "wd_cg_state_size")
    return n.value


def wd_cg_save_state(ctx) -> bytearray:
    """The CG state of a solve that stopped at maxit, as a host byte buffer."""
    buf = bytearray(wd_cg_state_size(ctx))
    cbuf = (ctypes.c_char * len(buf)).from_buffer(buf)
    _check(_lib.wd_cg_save_state(_P(ctx), ctypes.cast(cbuf, _P), len(buf)), "wd_cg_save_state")
    return buf


def cg_resume(ctx, state, src: torch.Tensor, x: torch.Tensor, tol: float, maxit: int):
    """Continue a saved CG state; x (output) receives the solution. Returns (status, iters, residual)."""
    for t in (src, x):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("src and x must be contiguous complex128 CUDA tensors")
    if src.numel() != x.numel():
        raise ValueError("cg_resume: src and x must have the same size")
    buf = bytes(state)
    it, res = ctypes.c_int(), ctypes.c_double()
    st = _lib.cg_resume(_P(ctx), ctypes.c_char_p(buf), len(buf), _P(_ptr(src)), _P(_ptr(x)), float(tol), int(maxit),
                        ctypes.byref(it), ctypes.byref(res))
    _check(st, "cg_resume", allow=(WD_OK, WD_NOT_CONVERGED, WD_BREAKDOWN))
    return st, it.value, res.value


def wd_generate_gauge(ctx, eps: float, seed: int, compress12: bool = False, U_out: torch.Tensor = None) -> None:
    if U_out is not None and (U_out.dtype != torch.complex128 or not U_out.is_cuda or not U_out.is_contiguous()):
        raise ValueError("U_out must be a contiguous complex128 CUDA tensor")
    _check(_lib.wd_generate_gauge(_P(ctx), float(eps), int(seed) & 0xFFFFFFFFFFFFFFFF, int(bool(compress12)),
                                  _P(_ptr(U_out)) if U_out is not None else None), "wd_generate_gauge")


def wd_generate_source(ctx, seed: int, out: torch.Tensor) -> None:
    if out.dtype != torch.complex128 or not out.is_cuda or not out.is_contiguous():
        raise ValueError("out must be a contiguous complex128 CUDA tensor")
    _check(_lib.wd_generate_source(_P(ctx), int(seed) & 0xFFFFFFFFFFFFFFFF, _P(_ptr(out))), "wd_generate_source")


def wd_coo_build(ctx, U: torch.Tensor):
    """D in the paper's coordinate format: returns (row int32, col int32, val complex128) device tensors."""
    if U.dtype != torch.complex128 or not U.is_cuda or not U.is_contiguous():
        raise ValueError("U must be a contiguous complex128 CUDA tensor")
    V = U.numel() // 36
    n = 49 * 12 * V
    row = torch.empty(n, dtype=torch.int32, device=U.device)
    col = torch.empty(n, dtype=torch.int32, device=U.device)
    val = torch.empty(n, dtype=torch.complex128, device=U.device)
    nnz = ctypes.c_longlong()
    _check(_lib.wd_coo_build(_P(ctx), _P(_ptr(U)), _P(_ptr(row)), _P(_ptr(col)), _P(_ptr(val)), n,
                             ctypes.byref(nnz)), "wd_coo_build")
    return row, col, val


def wd_coo_spmv(ctx, row, col, val, inp: torch.Tensor, out: torch.Tensor) -> None:
    _check(_lib.wd_coo_spmv(_P(ctx), row.numel(), _P(_ptr(row)), _P(_ptr(col)), _P(_ptr(val)), _P(_ptr(inp)),
                            _P(_ptr(out))), "wd_coo_spmv")


def _check_multi(t: torch.Tensor, name: str) -> int:
    if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() or t.dim() != 7:
        raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor [nrhs, Lt, Lz, Ly, Lx, 4, 3]")
    return t.shape[0]


def wd_apply_multi(ctx, inp: torch.Tensor, out: torch.Tensor, dagger: bool = False) -> None:
    n = _check_multi(inp, "inp")
    _check_multi(out, "out")
    _check(_lib.wd_apply_multi(_P(ctx), _P(_ptr(inp)), _P(_ptr(out)), n, int(bool(dagger))), "wd_apply_multi")


def cg_solve_multi(ctx, src: torch.Tensor, x: torch.Tensor, tol: float, maxit: int):
    """Returns (status, iterations per RHS, true relative residual per RHS); x updated in place."""
    n = _check_multi(src, "src")
    _check_multi(x, "x")
    it = (_I * n)()
    res = (_D * n)()
    st = _lib.cg_solve_multi(_P(ctx), _P(_ptr(src)), _P(_ptr(x)), n, float(tol), int(maxit), it, res)
    _check(st, "cg_solve_multi", allow=(WD_OK, WD_NOT_CONVERGED, WD_BREAKDOWN))
    return st, list(it), list(res)


def wd_get_multi_stats(ctx) -> dict:
    s = WdMultiStats()
    _check(_lib.wd_get_multi_stats(_P(ctx), ctypes.byref(s)), "wd_get_multi_stats")
    return {name: getattr(s, name) for name, _ in WdMultiStats._fields_}


def wd_dslash_noalloc(dims, kappa: float, U: torch.Tensor, inp: torch.Tensor, out: torch.Tensor,
                      dagger: bool = False, norm2_out: torch.Tensor = None, boundary=(1, 1, 1, -1),
                      stream=None) -> None:
    """out = D inp (or D^dagger inp) without any device allocation; all tensors on the device,
    canonical complex128 layouts; norm2_out: optional float64 device tensor of one element."""
    for t in (U, inp, out):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("U, inp and out must be contiguous complex128 CUDA tensors")
    if norm2_out is not None and (norm2_out.dtype != torch.float64 or not norm2_out.is_cuda):
        raise ValueError("norm2_out must be a float64 CUDA tensor")
    d = (_I * 4)(*[int(v) for v in dims])
    b = (_I * 4)(*[int(v) for v in boundary]) if boundary is not None else None
    _check(_lib.wd_dslash_noalloc(d, float(kappa), b, _P(_ptr(U)), _P(_ptr(inp)), _P(_ptr(out)),
                                  int(bool(dagger)),
                                  _P(_ptr(norm2_out)) if norm2_out is not None else None,
                                  _P(_stream_handle(stream))), "wd_dslash_noalloc")


def wd_set_option(ctx, key: int, value: float) -> None:
    _check(_lib.wd_set_option(_P(ctx), int(key), float(value)), "wd_set_option")


def wd_get_stats(ctx) -> dict:
    s = WdStats()
    _check(_lib.wd_get_stats(_P(ctx), ctypes.byref(s)), "wd_get_stats")
    return {name: getattr(s, name) for name, _ in WdStats._fields_}


def wd_get_residual_history(ctx, max_entries: int = 1 << 16) -> list:
    buf = (_D * max_entries)()
    n = _I(0)
    _check(_lib.wd_get_residual_history(_P(ctx), buf, int(max_entries), ctypes.byref(n)), "wd_get_residual_history")
    return list(buf[: n.value])


def wd_measure_fp64_peak(stream=None, repeats: int = 5) -> float:
    """FP64 FMA throughput of the current device in TFLOP/s (the FP64 compute ceiling)."""
    tf = _D(0.0)
    _check(_lib.wd_measure_fp64_peak(_P(_stream_handle(stream)), int(repeats), ctypes.byref(tf)),
           "wd_measure_fp64_peak")
    return tf.value


def wd_time_dslash(ctx, dagger: bool = False, launches: int = 20) -> float:
    ms = _D(0.0)
    _check(_lib.wd_time_dslash(_P(ctx), int(bool(dagger)), int(launches), ctypes.byref(ms)), "wd_time_dslash")
    return ms.value


# ------------------------------------------------------------------ convenience wrapper

class WilsonDirac:
    """A Wilson-Dirac operator on one lattice, bound to a CUDA stream.

    Fields are torch tensors in the canonical layout ``[Lt, Lz, Ly, Lx, 4, 3]`` (spinors) and
    ``[Lt, Lz, Ly, Lx, 4, 3, 3]`` (links), complex128 (complex64 for ``apply`` at precision 32).
    """

    def __init__(self, dims, kappa, boundary=(1, 1, 1, -1), precision=WD_PREC_F64, stream=None,
                 device="cuda"):
        self.dims = tuple(int(d) for d in dims)
        self.kappa = float(kappa)
        self.boundary = tuple(boundary)
        self.precision = int(precision)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = wd_create(self.dims, self.kappa, self.boundary, self.precision, self.stream)
        lx, ly, lz, lt = self.dims
        self.spinor_shape = (lt, lz, ly, lx, 4, 3)

    def close(self):
        if getattr(self, "ctx", None):
            wd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_kappa(self, kappa):
        wd_set_kappa(self.ctx, kappa)
        self.kappa = float(kappa)

    def load_gauge(self, U, compress12=False, check=True) -> float:
        return wd_load_gauge(self.ctx, U.contiguous(), compress12, check)

    def _spinor_numel(self):
        n = 12
        for d in self.dims:
            n *= d
        return n

    def apply(self, psi, dagger=False, out=None):
        want = torch.complex64 if (self.precision & ~WD_EVEN_ODD) == WD_PREC_F32 else torch.complex128
        if psi.dtype != want or psi.numel() != self._spinor_numel():
            raise ValueError(f"apply: psi must be a {want} spinor field of shape {self.spinor_shape}")
        if out is None:
            out = torch.empty_like(psi)
        wd_apply(self.ctx, psi.contiguous(), out, dagger)
        return out

    def solve(self, src, x0=None, tol=1e-10, maxit=2000):
        if src.numel() != self._spinor_numel() or (x0 is not None and x0.numel() != src.numel()):
            raise ValueError(f"solve: src (and x0) must be spinor fields of shape {self.spinor_shape}")
        x = torch.zeros_like(src) if x0 is None else x0.clone()
        status, iters, res = cg_solve(self.ctx, src.contiguous(), x, tol, maxit)
        return x, iters, res, status

    def save_state(self) -> bytearray:
        """The state of the last solve, which must have stopped at maxit (WD_NOT_CONVERGED)."""
        return wd_cg_save_state(self.ctx)

    def resume(self, state, src, tol=1e-10, maxit=2000):
        """Continue a saved solve; maxit counts the iterations before the save too."""
        if src.numel() != self._spinor_numel():
            raise ValueError(f"resume: src must be a spinor field of shape {self.spinor_shape}")
        x = torch.empty_like(src)
        status, iters, res = cg_resume(self.ctx, state, src.contiguous(), x, tol, maxit)
        return x, iters, res, status

    def set_option(self, key, value):
        wd_set_option(self.ctx, key, value)

    def stats(self):
        return wd_get_stats(self.ctx)

    def residual_history(self, max_entries: int = 1 << 16):
        return wd_get_residual_history(self.ctx, max_entries)

    def time_dslash(self, dagger=False, launches=20) -> float:
        return wd_time_dslash(self.ctx, dagger, launches)

    def generate_gauge(self, eps, seed, compress12=False, return_field=False):
        lx, ly, lz, lt = self.dims
        U = torch.empty((lt, lz, ly, lx, 4, 3, 3), dtype=torch.complex128, device=self.device) if return_field else None
        wd_generate_gauge(self.ctx, eps, seed, compress12, U)
        return U

    def generate_source(self, seed):
        out = torch.empty(self.spinor_shape, dtype=torch.complex128, device=self.device)
        wd_generate_source(self.ctx, seed, out)
        return out

    def apply_multi(self, psi, dagger=False, out=None):
        if out is None:
            out = torch.empty_like(psi)
        wd_apply_multi(self.ctx, psi.contiguous(), out, dagger)
        return out

    def solve_multi(self, src, x0=None, tol=1e-10, maxit=2000):
        x = torch.zeros_like(src) if x0 is None else x0.clone()
        status, iters, res = cg_solve_multi(self.ctx, src.contiguous(), x, tol, maxit)
        return x, iters, res, status

    def multi_stats(self):
        return wd_get_multi_stats(self.ctx)


# ------------------------------------------------------------------ serving

def _struct_dict(obj):
    return {name: getattr(obj, name) for name, _ in obj._fields_}


class Server:
    """Persistent solve server (wd_server_*): continuous admission of single-RHS requests."""

    def __init__(self, budget_bytes: float, slots: int = 4, max_batch: int = None):
        h = _P()
        _check(_lib.wd_server_create(float(budget_bytes), int(slots), ctypes.byref(h)), "wd_server_create")
        self.h = h.value
        self._keep = {}
        if max_batch is not None:
            self.set_max_batch(max_batch)

    def set_max_batch(self, max_batch: int):
        _check(_lib.wd_server_set_max_batch(_P(self.h), int(max_batch)), "wd_server_set_max_batch")

    def set_policy(self, policy: int, max_wait_ms: float = 1000.0):
        """0: oldest request first; 1: least estimated work first, the oldest first once it has
        waited more than max_wait_ms."""
        _check(_lib.wd_server_set_policy(_P(self.h), int(policy), float(max_wait_ms)), "wd_server_set_policy")

    def submit(self, dims, kappa, eps, gauge_seed, source_seed, tol, precision=WD_PREC_MIXED_F32, maxit=20000,
               boundary=None, src_host: torch.Tensor = None, x_host: torch.Tensor = None) -> int:
        r = WdRequest()
        for i in range(4):
            r.dims[i] = int(dims[i])
        r.kappa, r.eps, r.tol = float(kappa), float(eps), float(tol)
        r.gauge_seed = int(gauge_seed) & 0xFFFFFFFFFFFFFFFF
        r.source_seed = int(source_seed) & 0xFFFFFFFFFFFFFFFF
        r.maxit, r.precision = int(maxit), int(precision)
        if boundary is not None:
            r.boundary_set = 1
            for i in range(4):
                r.boundary[i] = int(boundary[i])
        for t in (src_host, x_host):
            if t is not None and (t.is_cuda or t.dtype != torch.complex128 or not t.is_contiguous()):
                raise ValueError("src_host / x_host must be contiguous complex128 CPU tensors")
        r.src_host = src_host.data_ptr() if src_host is not None else None
        r.x_host = x_host.data_ptr() if x_host is not None else None
        rid = ctypes.c_longlong()
        _check(_lib.wd_server_submit(_P(self.h), ctypes.byref(r), ctypes.byref(rid)), "wd_server_submit")
        self._keep[rid.value] = (src_host, x_host)
        return rid.value

    def wait(self, rid: int) -> dict:
        res = WdResult()
        _check(_lib.wd_server_wait(_P(self.h), ctypes.c_longlong(rid), ctypes.byref(res)), "wd_server_wait")
        self._keep.pop(rid, None)
        return _struct_dict(res)

    def poll(self, rid: int):
        res = WdResult()
        done = _I(0)
        _check(_lib.wd_server_poll(_P(self.h), ctypes.c_longlong(rid), ctypes.byref(res), ctypes.byref(done)),
               "wd_server_poll")
        if done.value:
            self._keep.pop(rid, None)
            return _struct_dict(res)
        return None

    def stats(self) -> dict:
        s = WdServerStats()
        _check(_lib.wd_server_get_stats(_P(self.h), ctypes.byref(s)), "wd_server_get_stats")
        return _struct_dict(s)

    def close(self):
        if getattr(self, "h", None):
            _lib.wd_server_destroy(_P(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
