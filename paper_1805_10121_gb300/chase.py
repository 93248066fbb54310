"""Thin ctypes binding to libchase.so (the C ABI declared in include/chase.h).

Argument marshalling only: every function passes the data pointers of torch
tensors (device or host) and the sizes to the C entry point of the same
name; all arithmetic runs in the library's kernels.  Importing this module
does not load the library; the first call does, and fails loudly if the
library has not been built.
"""

from __future__ import annotations

import contextlib
import ctypes
import os
import re
from typing import Optional

import numpy as np
import torch

__all__ = [
    "ChaseError", "ChaseOpts", "ChaseStats", "lib", "lib_path", "declared_symbols",
    "chase_opts_default", "chase_last_error", "chase_filter_mixed", "chase_kernel_launches", "chase_device_allocations",
    "chase_kernel_timing",
    "chase_kernel_timing_read", "chase_wait_selftest", "CHASE_TIMED_SPLIT_PRODUCT", "CHASE_TIMED_FP64_PRODUCT", "chase_filter", "chase_lanczos",
    "chase_degrees", "chase_lock", "chase_tridiag_eigh", "chase_dos_estimate", "chase_orthonormalize",
    "chase_rayleigh_ritz", "chase_residuals", "chase_residuals_noalloc", "chase_solve",
    "CHASE_OK", "CHASE_INVALID_ARG", "CHASE_NOT_CONVERGED", "CHASE_QR_BREAKDOWN",
    "CHASE_BOUND_VIOLATION", "CHASE_CUDA_ERROR", "CHASE_OUT_OF_MEMORY", "CHASE_TIMEOUT",
    "CHASE_EIGENSOLVER_ERROR", "CHASE_CONV_ABS", "CHASE_CONV_REL", "CHASE_FP64",
    "CHASE_SPLIT_BF16", "CHASE_SPLIT_BF16_RR", "CHASE_SPLIT_BF16_ADAPT",
    "CHASE_SPLIT_BF16_4", "CHASE_SPLIT_BF16_3", "CHASE_TILE_AUTO", "CHASE_STORAGE_FULL",
    "CHASE_STORAGE_LOWER", "ChaseBatchStats", "chase_filter_batched",
    "chase_solve_batched", "chase_filter_real", "chase_residuals_real", "chase_solve_real",
    "chase_filter_c32", "chase_filter_f32", "chase_residuals_c32", "chase_residuals_f32",
    "chase_solve_c32", "chase_solve_f32",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
_HEADER = os.path.join(os.path.dirname(_PKG), "include", "chase.h")

CHASE_OK = 0
CHASE_INVALID_ARG = 1
CHASE_NOT_CONVERGED = 2
CHASE_QR_BREAKDOWN = 3
CHASE_BOUND_VIOLATION = 4
CHASE_CUDA_ERROR = 5
CHASE_OUT_OF_MEMORY = 6
CHASE_TIMEOUT = 7
CHASE_EIGENSOLVER_ERROR = 8
CHASE_FP64 = 0
CHASE_SPLIT_BF16 = 1
CHASE_SPLIT_BF16_RR = 2
CHASE_SPLIT_BF16_ADAPT = 3
CHASE_SPLIT_BF16_4 = 4
CHASE_SPLIT_BF16_3 = 5
CHASE_CONV_ABS = 0
CHASE_CONV_REL = 1
CHASE_TILE_AUTO = -1
CHASE_STORAGE_FULL = 0
CHASE_STORAGE_LOWER = 1


class ChaseError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


class ChaseOpts(ctypes.Structure):
    _fields_ = [
        ("deg", ctypes.c_int), ("optim", ctypes.c_int), ("deg_extra", ctypes.c_int),
        ("deg_max", ctypes.c_int), ("max_iter", ctypes.c_int), ("lanczos_iter", ctypes.c_int),
        ("num_lanczos", ctypes.c_int), ("approx", ctypes.c_int), ("dos_sigma", ctypes.c_double),
        ("conv_mode", ctypes.c_int), ("precision", ctypes.c_int), ("storage", ctypes.c_int),
    ]


class ChaseStats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("nconv", ctypes.c_int),
        ("matvecs", ctypes.c_longlong), ("filter_matvecs", ctypes.c_longlong),
        ("b_sup", ctypes.c_double), ("mu1", ctypes.c_double), ("mu_nevnex", ctypes.c_double),
        ("tol_eff", ctypes.c_double), ("flops_filter", ctypes.c_double),
        ("flops_total", ctypes.c_double), ("t_total", ctypes.c_double),
        ("t_lanczos", ctypes.c_double), ("t_filter", ctypes.c_double), ("t_qr", ctypes.c_double),
        ("t_rr", ctypes.c_double), ("t_eigh", ctypes.c_double), ("t_resid", ctypes.c_double),
        ("t_host", ctypes.c_double), ("t_rr_product", ctypes.c_double),
        ("flops_rr_product", ctypes.c_double), ("filter_slices_low", ctypes.c_int),
        ("lanczos_matvecs", ctypes.c_longlong), ("filter_matvecs_low", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ChaseBatchStats(ctypes.Structure):
    _fields_ = [
        ("problems", ctypes.c_int), ("steps", ctypes.c_int), ("tile_config", ctypes.c_int),
        ("launches", ctypes.c_int), ("matvecs", ctypes.c_longlong), ("flops", ctypes.c_double),
        ("t_autotune", ctypes.c_double), ("t_graph_build", ctypes.c_double),
        ("t_steps", ctypes.c_double), ("t_product", ctypes.c_double), ("t_total", ctypes.c_double),
        ("t_qr", ctypes.c_double), ("t_rr", ctypes.c_double), ("t_eigh", ctypes.c_double),
        ("t_lock", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_c_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

_SIGNATURES = {
    "chase_opts_default": (_int, [ctypes.POINTER(ChaseOpts)]),
    "chase_last_error": (ctypes.c_char_p, []),
    "chase_kernel_launches": (ctypes.c_longlong, []),
    "chase_device_allocations": (ctypes.c_longlong, []),
    "chase_kernel_timing": (_int, [_int]),
    "chase_wait_selftest": (_int, [ctypes.c_longlong, _c_p]),
    "chase_kernel_timing_read": (_int, [_int, _dp, ctypes.POINTER(ctypes.c_longlong), _dp, _dp]),
    "chase_filter": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _c_p, _dbl, _dbl, _dbl, _int, _c_p,
                            _c_p]),
    "chase_filter_mixed": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _c_p, _c_p, _dbl, _dbl,
                                  _dbl, _c_p, _c_p]),
    "chase_filter_batched": (_int, [_int, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p,
                                    _c_p, _int, _int, ctypes.POINTER(ChaseBatchStats), _c_p]),
    "chase_solve_batched": (_int, [_int, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p,
                                   _c_p, ctypes.POINTER(ChaseOpts), _c_p, _c_p,
                                   ctypes.POINTER(ChaseBatchStats), _c_p]),
    "chase_lanczos": (_int, [_c_p, _i64, _i64, _int, _int, _int, _int, _int, _dbl, _c_p, _c_p,
                             _i64, _dp, _dp, _dp, _dp, _c_p]),
    "chase_degrees": (_int, [_int, _dp, _dp, _dbl, _dbl, _dbl, _int, _int, _ip]),
    "chase_lock": (_int, [_int, _dp, _dp, _dbl, _ip, _ip]),
    "chase_tridiag_eigh": (_int, [_int, _dp, _dp, _dp, _dp]),
    "chase_dos_estimate": (_int, [_int, _ip, _dp, _dp, _dbl, _dbl, _dbl, _dbl, _dp, _ip]),
    "chase_orthonormalize": (_int, [_c_p, _i64, _i64, _int, _c_p, _i64, _int, _c_p]),
    "chase_rayleigh_ritz": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _dp, _dp, _c_p]),
    "chase_residuals": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _dp, _dp, _c_p]),
    "chase_residuals_noalloc": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _c_p, _c_p, _c_p]),
    "chase_filter_real": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _c_p, _dbl, _dbl, _dbl, _int,
                                 _c_p, _c_p]),
    "chase_residuals_real": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _dp, _dp, _c_p]),
    "chase_solve_real": (_int, [_c_p, _i64, _i64, _int, _int, _dbl, _c_p, _i64, _dp, _dp, _c_p,
                                ctypes.POINTER(ChaseOpts), ctypes.POINTER(ChaseStats), _c_p]),
    "chase_filter_c32": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _c_p, _dbl, _dbl, _dbl, _c_p,
                                _c_p]),
    "chase_filter_f32": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _c_p, _dbl, _dbl, _dbl, _c_p,
                                _c_p]),
    "chase_residuals_c32": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _dp, _dp, _c_p]),
    "chase_residuals_f32": (_int, [_c_p, _i64, _i64, _c_p, _i64, _int, _dp, _dp, _c_p]),
    "chase_solve_c32": (_int, [_c_p, _i64, _i64, _int, _int, _dbl, _c_p, _i64, _dp, _dp, _c_p,
                               ctypes.POINTER(ChaseOpts), ctypes.POINTER(ChaseStats), _c_p]),
    "chase_solve_f32": (_int, [_c_p, _i64, _i64, _int, _int, _dbl, _c_p, _i64, _dp, _dp, _c_p,
                               ctypes.POINTER(ChaseOpts), ctypes.POINTER(ChaseStats), _c_p]),
    "chase_solve": (_int, [_c_p, _i64, _i64, _int, _int, _dbl, _c_p, _i64, _dp, _dp, _c_p,
                           ctypes.POINTER(ChaseOpts), ctypes.POINTER(ChaseStats), _c_p]),
}

_lib = None


def lib_path() -> str:
    return os.path.join(_PKG, "libchase.so")


def lib() -> ctypes.CDLL:
    """Load libchase.so (built in-tree by ``paper_1805_10121_gb300.build``)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
        handle = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def declared_symbols(header: str = _HEADER) -> list[str]:
    """Names of the functions declared in include/chase.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chase_[a-z_0-9]+)\s*\(", text)))


def chase_kernel_launches() -> int:
    return int(lib().chase_kernel_launches())


def chase_device_allocations() -> int:
    return int(lib().chase_device_allocations())


CHASE_TIMED_SPLIT_PRODUCT = 0
CHASE_TIMED_FP64_PRODUCT = 1


def chase_kernel_timing(enable: bool) -> None:
    """Start (clearing the record) or stop the library's product-kernel timing."""
    _check(lib().chase_kernel_timing(1 if enable else 0), "chase_kernel_timing")


def chase_kernel_timing_read(kind: int) -> dict:
    """Summed CUDA-event time, launches and FLOPs of the recorded product
    launches of one kind (CHASE_TIMED_SPLIT_PRODUCT or _FP64_PRODUCT)."""
    s, f, tf = np.zeros(1), np.zeros(1), np.zeros(1)
    n = ctypes.c_longlong(0)
    _check(lib().chase_kernel_timing_read(int(kind), _dptr(s), ctypes.byref(n), _dptr(f), _dptr(tf)),
           "chase_kernel_timing_read")
    return {"seconds": float(s[0]), "launches": int(n.value), "flops": float(f[0]),
            "tensor_flops": float(tf[0])}


def chase_wait_selftest(budget_cycles: int, stream=None) -> int:
    """Run the kernels' bounded mbarrier wait on a barrier nothing arrives
    at; returns the status (CHASE_TIMEOUT when the wait gave up)."""
    s = ctypes.c_void_p(0 if stream is None else int(stream))
    if stream is None and torch.cuda.is_available():
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return int(lib().chase_wait_selftest(int(budget_cycles), s))


def chase_last_error() -> str:
    return (lib().chase_last_error() or b"").decode()


def _check(status: int, where: str, allow=(CHASE_OK,)):
    if status not in allow:
        raise ChaseError(status, where, chase_last_error())
    return status


def _mat(t: torch.Tensor, rows: int, name: str, dtype=torch.complex128):
    """Pointer and leading dimension of a column-major complex128 (or, for
    the real entry points, float64) matrix."""
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if t.dim() != 2 or t.shape[0] != rows:
        raise ValueError(f"{name} must have {rows} rows")
    if t.shape[1] > 1 and t.stride(0) != 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    ld = t.stride(1) if t.shape[1] > 1 else max(rows, 1)
    if t.shape[1] == 1 and t.stride(0) != 1:
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr()), ld


def _stream(t: torch.Tensor, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if t.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(0)


def _f64(a, n: Optional[int] = None) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and x.shape != (n,):
        raise ValueError(f"expected {n} values")
    return x


def _dptr(x: np.ndarray):
    return x.ctypes.data_as(_dp)


def _iptr(x: np.ndarray):
    return x.ctypes.data_as(_ip)


def chase_opts_default(**overrides) -> ChaseOpts:
    o = ChaseOpts()
    _check(lib().chase_opts_default(ctypes.byref(o)), "chase_opts_default")
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _filter(entry, dtype, H, V, degrees, b_sup, mu1, mu_nevnex, work, stream, precision):
    n = H.shape[0]
    hp, ldh = _mat(H, n, "H", dtype)
    vp, ldv = _mat(V, n, "V", dtype)
    b = V.shape[1]
    if isinstance(degrees, torch.Tensor):
        if degrees.dtype != torch.int32 or not degrees.is_contiguous():
            raise TypeError("degrees must be a contiguous int32 tensor")
        deg_keep = degrees
        dptr = ctypes.c_void_p(degrees.data_ptr())
    else:
        deg_keep = np.ascontiguousarray(np.asarray(degrees, dtype=np.int32))
        dptr = ctypes.c_void_p(deg_keep.ctypes.data)
    if len(deg_keep) != b:
        raise ValueError("one degree per column")
    wp = ctypes.c_void_p(work.data_ptr()) if work is not None else None
    args = [hp, n, ldh, vp, ldv, b, dptr, float(b_sup), float(mu1), float(mu_nevnex)]
    if precision is not None:
        args.append(int(precision))
    st = getattr(lib(), entry)(*args, wp, _stream(V, stream))
    _check(st, entry)
    return V


def chase_filter(H, V, degrees, b_sup, mu1, mu_nevnex, work=None, stream=None,
                 precision=CHASE_FP64):
    """Filter the columns of V in place (Alg. 4).  ``degrees``: int32 tensor
    (host or device) or a sequence of ints."""
    return _filter("chase_filter", torch.complex128, H, V, degrees, b_sup, mu1, mu_nevnex, work,
                   stream, precision)


def chase_filter_mixed(H, V, degrees, slices, b_sup, mu1, mu_nevnex, work=None, stream=None):
    """Alg. 4 with a precision per column: ``slices[a]`` in {3, 4, 7} slices of
    the split-BF16 product for column a (complex128 tensors, V in place)."""
    n = H.shape[0]
    hp, ldh = _mat(H, n, "H")
    vp, ldv = _mat(V, n, "V")
    b = V.shape[1]
    deg = np.ascontiguousarray(np.asarray(degrees, dtype=np.int32))
    ns = np.ascontiguousarray(np.asarray(slices, dtype=np.int32))
    if deg.shape != (b,) or ns.shape != (b,):
        raise ValueError("one degree and one slice count per column")
    wp = ctypes.c_void_p(work.data_ptr()) if work is not None else None
    _check(lib().chase_filter_mixed(hp, n, ldh, vp, ldv, b, ctypes.c_void_p(deg.ctypes.data),
                                    ctypes.c_void_p(ns.ctypes.data), float(b_sup), float(mu1),
                                    float(mu_nevnex), wp, _stream(V, stream)),
           "chase_filter_mixed")
    return V


def chase_filter_c32(H, V, degrees, b_sup, mu1, mu_nevnex, work=None, stream=None):
    """Alg. 4 in single precision (complex64 tensors)."""
    return _filter("chase_filter_c32", torch.complex64, H, V, degrees, b_sup, mu1, mu_nevnex,
                   work, stream, None)


def chase_filter_f32(H, V, degrees, b_sup, mu1, mu_nevnex, work=None, stream=None):
    """Alg. 4 in single precision for a real symmetric H (float32 tensors)."""
    return _filter("chase_filter_f32", torch.float32, H, V, degrees, b_sup, mu1, mu_nevnex, work,
                   stream, None)


def chase_filter_real(H, V, degrees, b_sup, mu1, mu_nevnex, work=None, stream=None,
                      precision=CHASE_FP64):
    """Alg. 4 for a real symmetric H (float64 tensors)."""
    return _filter("chase_filter_real", torch.float64, H, V, degrees, b_sup, mu1, mu_nevnex, work,
                   stream, precision)


def chase_filter_batched(Hs, Vs, degrees, b_sup, mu1, mu_nevnex, precision=CHASE_FP64,
                         tile=CHASE_TILE_AUTO, stream=None):
    """Filter every V[p] in place with its own H[p], degrees and bounds, all
    problems in one grouped launch per degree step.  ``Hs``, ``Vs``: lists
    of column-major complex128 device tensors; ``degrees``: list of int
    sequences.  Returns the call's counters and times as a dict."""
    P = len(Hs)
    if not (len(Vs) == len(degrees) == P):
        raise ValueError("one V and one degree list per H")
    hp = (ctypes.c_void_p * max(P, 1))()
    vp = (ctypes.c_void_p * max(P, 1))()
    dp = (ctypes.c_void_p * max(P, 1))()
    n = np.zeros(max(P, 1), dtype=np.int64)
    ldh = np.ones(max(P, 1), dtype=np.int64)
    ldv = np.ones(max(P, 1), dtype=np.int64)
    b = np.zeros(max(P, 1), dtype=np.int32)
    keep = []
    for p in range(P):
        H, V = Hs[p], Vs[p]
        n[p] = H.shape[0]
        hp[p], ldh[p] = _mat(H, int(n[p]), "H")
        vp[p], ldv[p] = _mat(V, int(n[p]), "V")
        b[p] = V.shape[1]
        d = np.ascontiguousarray(np.asarray(degrees[p], dtype=np.int32))
        if d.shape != (int(b[p]),):
            raise ValueError("one degree per column")
        keep.append(d)
        dp[p] = d.ctypes.data
    bs, m1, mn = _f64(b_sup, P), _f64(mu1, P), _f64(mu_nevnex, P)
    stats = ChaseBatchStats()
    st = lib().chase_filter_batched(
        P, ctypes.cast(hp, _c_p), n.ctypes.data, ldh.ctypes.data, ctypes.cast(vp, _c_p),
        ldv.ctypes.data, b.ctypes.data, ctypes.cast(dp, _c_p), bs.ctypes.data, m1.ctypes.data,
        mn.ctypes.data, int(precision), int(tile), ctypes.byref(stats),
        _stream(Vs[0], stream) if P else ctypes.c_void_p(0 if stream is None else int(stream)))
    _check(st, "chase_filter_batched")
    return stats.as_dict()


def chase_solve_batched(Hs, nev, nex, tol, Vs, lanczos_starts, opts=None, stream=None):
    """ChASE on every problem of the batch with grouped filters.  ``Hs``,
    ``Vs``, ``lanczos_starts``: lists of column-major complex128 device
    tensors; ``nev``, ``nex``, ``tol``: one value per problem (or a scalar).
    Returns (status, statuses, [Lambda], [resid], [stats], batch_stats)."""
    P = len(Hs)
    if not (len(Vs) == len(lanczos_starts) == P):
        raise ValueError("one V and one start block per H")
    nev = np.broadcast_to(np.asarray(nev, dtype=np.int32), (P,)).copy()
    nex = np.broadcast_to(np.asarray(nex, dtype=np.int32), (P,)).copy()
    tol = np.broadcast_to(np.asarray(tol, dtype=np.float64), (P,)).copy()
    m = max(P, 1)
    hp, vp, sp = (ctypes.c_void_p * m)(), (ctypes.c_void_p * m)(), (ctypes.c_void_p * m)()
    lp, rp = (ctypes.c_void_p * m)(), (ctypes.c_void_p * m)()
    n = np.zeros(m, dtype=np.int64)
    ldh = np.ones(m, dtype=np.int64)
    ldv = np.ones(m, dtype=np.int64)
    lams, res = [], []
    for p in range(P):
        n[p] = Hs[p].shape[0]
        hp[p], ldh[p] = _mat(Hs[p], int(n[p]), "H")
        vp[p], ldv[p] = _mat(Vs[p], int(n[p]), "V")
        sp[p], lds = _mat(lanczos_starts[p], int(n[p]), "lanczos_starts")
        if lds != n[p] and lanczos_starts[p].shape[1] > 1:
            raise ValueError("lanczos_starts must have leading dimension N")
        nx = int(nev[p] + nex[p])
        if Vs[p].shape[1] != nx:
            raise ValueError("V must have nev + nex columns")
        lams.append(np.zeros(nx))
        res.append(np.zeros(nx))
        lp[p] = lams[-1].ctypes.data
        rp[p] = res[-1].ctypes.data
    if opts is None:
        opts = chase_opts_default()
    statuses = np.zeros(m, dtype=np.int32)
    stats = (ChaseStats * m)()
    bstats = ChaseBatchStats()
    st = lib().chase_solve_batched(
        P, ctypes.cast(hp, _c_p), n.ctypes.data, ldh.ctypes.data, nev.ctypes.data,
        nex.ctypes.data, tol.ctypes.data, ctypes.cast(vp, _c_p), ldv.ctypes.data,
        ctypes.cast(lp, _c_p), ctypes.cast(rp, _c_p), ctypes.cast(sp, _c_p), ctypes.byref(opts),
        statuses.ctypes.data, ctypes.cast(stats, _c_p), ctypes.byref(bstats),
        _stream(Vs[0], stream) if P else ctypes.c_void_p(0 if stream is None else int(stream)))
    _check(st, "chase_solve_batched",
           allow=(CHASE_OK, CHASE_NOT_CONVERGED, CHASE_BOUND_VIOLATION))
    return (st, statuses[:P].tolist(), lams, res, [stats[p].as_dict() for p in range(P)],
            bstats.as_dict())


def chase_lanczos(H, k, nvec, approx, nev, nex, starts, V=None, dos_sigma=0.25, stream=None):
    n = H.shape[0]
    hp, ldh = _mat(H, n, "H")
    sp, lds = _mat(starts, n, "starts")
    if lds != max(n, 1) and starts.shape[1] > 1:
        raise ValueError("starts must have leading dimension N")
    vp, ldv = (None, n) if V is None else _mat(V, n, "V")
    out = np.zeros(4)
    st = lib().chase_lanczos(hp, n, ldh, int(k), int(nvec), int(approx), int(nev), int(nex),
                             float(dos_sigma), sp, vp, ldv, _dptr(out[0:]), _dptr(out[1:]),
                             _dptr(out[2:]), _dptr(out[3:]), _stream(H, stream))
    _check(st, "chase_lanczos")
    res = {"b_sup": out[0], "theta_absmax": out[3]}
    if not approx:
        res.update(mu1=out[1], mu_nevnex=out[2])
    return res


def chase_degrees(resid, ritz, c, e, tol, deg_extra=2, deg_max=36):
    r = _f64(resid)
    lam = _f64(ritz, len(r))
    out = np.zeros(len(r), dtype=np.int32)
    _check(lib().chase_degrees(len(r), _dptr(r), _dptr(lam), float(c), float(e), float(tol),
                               int(deg_extra), int(deg_max), _iptr(out)), "chase_degrees")
    return out


def chase_lock(ritz, resid, tol):
    lam = _f64(ritz)
    r = _f64(resid, len(lam))
    order = np.zeros(len(lam), dtype=np.int32)
    n = ctypes.c_int(0)
    _check(lib().chase_lock(len(lam), _dptr(lam), _dptr(r), float(tol), _iptr(order),
                            ctypes.byref(n)), "chase_lock")
    return order, n.value


def chase_tridiag_eigh(diag, off):
    dg = _f64(diag)
    k = len(dg)
    of = _f64(off, max(k - 1, 0)) if k > 1 else np.zeros(1)
    w = np.zeros(k)
    z = np.zeros(k * k)
    _check(lib().chase_tridiag_eigh(k, _dptr(dg), _dptr(of), _dptr(w), _dptr(z)),
           "chase_tridiag_eigh")
    return w, z.reshape(k, k).T.copy()


def chase_dos_estimate(nodes, target, mu1, b_sup, dos_sigma=0.25):
    """mu_nev+nex of Alg. 6 line 11 from per-run (theta, weights) pairs.
    Returns ``(mu, halvings)``; ``halvings`` is -1 for the uniform fallback."""
    steps = np.array([len(th) for th, _ in nodes], dtype=np.int32)
    theta = _f64(np.concatenate([np.asarray(th, dtype=np.float64) for th, _ in nodes]))
    w = _f64(np.concatenate([np.asarray(x, dtype=np.float64) for _, x in nodes]))
    if w.shape != theta.shape:
        raise ValueError("one weight per Ritz value")
    mu = np.zeros(1)
    h = np.zeros(1, dtype=np.int32)
    _check(lib().chase_dos_estimate(len(nodes), _iptr(steps), _dptr(theta), _dptr(w),
                                    float(target), float(mu1), float(b_sup), float(dos_sigma),
                                    _dptr(mu), _iptr(h)), "chase_dos_estimate")
    return float(mu[0]), int(h[0])


def chase_orthonormalize(Y, V, stream=None):
    n = V.shape[0]
    vp, ldv = _mat(V, n, "V")
    if Y is None or Y.shape[1] == 0:
        yp, ldy, nconv = None, n, 0
    else:
        yp, ldy = _mat(Y, n, "Y")
        nconv = Y.shape[1]
    _check(lib().chase_orthonormalize(yp, n, ldy, nconv, vp, ldv, V.shape[1],
                                      _stream(V, stream)), "chase_orthonormalize")
    return V


def chase_rayleigh_ritz(H, Q, want_resid=True, stream=None):
    n = H.shape[0]
    hp, ldh = _mat(H, n, "H")
    qp, ldq = _mat(Q, n, "Q")
    b = Q.shape[1]
    ritz = np.zeros(b)
    resid = np.zeros(b) if want_resid else None
    _check(lib().chase_rayleigh_ritz(hp, n, ldh, qp, ldq, b, _dptr(ritz),
                                     _dptr(resid) if want_resid else None, _stream(Q, stream)),
           "chase_rayleigh_ritz")
    return ritz, resid


def _residuals(entry, dtype, H, V, lam, stream):
    n = H.shape[0]
    hp, ldh = _mat(H, n, "H", dtype)
    vp, ldv = _mat(V, n, "V", dtype)
    b = V.shape[1]
    lam = _f64(lam, b)
    out = np.zeros(b)
    _check(getattr(lib(), entry)(hp, n, ldh, vp, ldv, b, _dptr(lam), _dptr(out),
                                 _stream(V, stream)), entry)
    return out


def chase_residuals(H, V, lam, stream=None):
    return _residuals("chase_residuals", torch.complex128, H, V, lam, stream)


def chase_residuals_real(H, V, lam, stream=None):
    return _residuals("chase_residuals_real", torch.float64, H, V, lam, stream)


def chase_residuals_c32(H, V, lam, stream=None):
    return _residuals("chase_residuals_c32", torch.complex64, H, V, lam, stream)


def chase_residuals_f32(H, V, lam, stream=None):
    return _residuals("chase_residuals_f32", torch.float32, H, V, lam, stream)


def chase_residuals_noalloc(H, V, lam, resid, stream=None):
    """Residual norms into the device tensor ``resid`` (float64, b) from the
    device tensor ``lam``; the library allocates nothing for this call."""
    n = H.shape[0]
    hp, ldh = _mat(H, n, "H")
    vp, ldv = _mat(V, n, "V")
    b = V.shape[1]
    for t, name in ((lam, "lam"), (resid, "resid")):
        if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != b:
            raise ValueError(f"{name} must be a contiguous float64 tensor of {b} values")
    if any(t.device != V.device for t in (H, lam, resid)):
        raise ValueError("H, V, lam and resid must be on one device")
    ctx = torch.cuda.device(V.device) if V.is_cuda else contextlib.nullcontext()
    with ctx:
        _check(lib().chase_residuals_noalloc(hp, n, ldh, vp, ldv, b,
                                             ctypes.c_void_p(lam.data_ptr()),
                                             ctypes.c_void_p(resid.data_ptr()), _stream(V, stream)),
               "chase_residuals_noalloc")
    return resid


def _solve(entry, dtype, H, nev, nex, tol, V, lanczos_starts, Lambda, opts, stream,
           raise_not_converged):
    n = H.shape[0]
    nx = nev + nex
    hp, ldh = _mat(H, n, "H", dtype)
    vp, ldv = _mat(V, n, "V", dtype)
    sp, lds = _mat(lanczos_starts, n, "lanczos_starts", dtype)
    if lanczos_starts.shape[1] > 1 and lds != n:
        raise ValueError("lanczos_starts must have leading dimension N")
    lam = np.zeros(nx) if Lambda is None else np.array(Lambda, dtype=np.float64, copy=True)
    if lam.shape != (nx,):
        raise ValueError("Lambda must have nev + nex values")
    resid = np.zeros(nx)
    o = opts if opts is not None else chase_opts_default()
    stats = ChaseStats()
    st = getattr(lib(), entry)(hp, n, ldh, int(nev), int(nex), float(tol), vp, ldv, _dptr(lam),
                               _dptr(resid), sp, ctypes.byref(o), ctypes.byref(stats),
                               _stream(H, stream))
    allow = (CHASE_OK,) if raise_not_converged else (CHASE_OK, CHASE_NOT_CONVERGED)
    _check(st, entry, allow)
    return st, lam, resid, stats.as_dict()


def chase_solve(H, nev, nex, tol, V, lanczos_starts, Lambda=None, opts=None, stream=None,
                raise_not_converged=False):
    """Alg. 1.  V (N x (nev+nex)) is overwritten with the Ritz vectors.
    Returns ``(status, Lambda, resid, stats_dict)``."""
    return _solve("chase_solve", torch.complex128, H, nev, nex, tol, V, lanczos_starts, Lambda,
                  opts, stream, raise_not_converged)


def chase_solve_real(H, nev, nex, tol, V, lanczos_starts, Lambda=None, opts=None, stream=None,
                     raise_not_converged=False):
    """Alg. 1 for a real symmetric H (float64 tensors)."""
    return _solve("chase_solve_real", torch.float64, H, nev, nex, tol, V, lanczos_starts, Lambda,
                  opts, stream, raise_not_converged)


def chase_solve_c32(H, nev, nex, tol, V, lanczos_starts, Lambda=None, opts=None, stream=None,
                    raise_not_converged=False):
    """Alg. 1 in single precision (complex64 tensors)."""
    return _solve("chase_solve_c32", torch.complex64, H, nev, nex, tol, V, lanczos_starts, Lambda,
                  opts, stream, raise_not_converged)


def chase_solve_f32(H, nev, nex, tol, V, lanczos_starts, Lambda=None, opts=None, stream=None,
                    raise_not_converged=False):
    """Alg. 1 in single precision for a real symmetric H (float32 tensors)."""
    return _solve("chase_solve_f32", torch.float32, H, nev, nex, tol, V, lanczos_starts, Lambda,
                  opts, stream, raise_not_converged)
