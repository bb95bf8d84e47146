"""Python binding of libchol.so, the GB300 tiled Cholesky library.

Argument marshalling only: every function here forwards to the C entry point
of the same name declared in ``include/chol.h``; all computation runs in the
library's CUDA kernels.  There is no fallback: if ``libchol.so`` has not been
built (``python -m paper_2606_11937_gb300.build`` or
``__graft_entry__.build()``), the first call raises ``RuntimeError``.

Matrices are torch CUDA tensors in COLUMN-major layout (``t.stride(0) == 1``),
which is the library's convention (LAPACK, lower triangle).  ``colmajor(x)``
makes such a tensor from any 2-D tensor or numpy array.  Raw device pointers
(ints) are accepted wherever a tensor is.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchol.so")

# --------------------------------------------------------------------- constants
CHOL_OK, CHOL_ERR_ARG, CHOL_ERR_NOT_SPD, CHOL_ERR_NOMEM, CHOL_ERR_CUDA = 0, -1, -2, -3, -4
CHOL_ERR_TIMEOUT, CHOL_ERR_NOT_CONVERGED, CHOL_ERR_BUSY, CHOL_ERR_HANDLE, CHOL_ERR_UNSUPPORTED = -5, -6, -7, -8, -9
CHOL_FP64, CHOL_FP32, CHOL_TF32, CHOL_BF16, CHOL_FP16 = 0, 1, 2, 3, 4
CHOL_SCHED_AUTO, CHOL_SCHED_FORK_JOIN, CHOL_SCHED_FORK_JOIN_NAIVE, CHOL_SCHED_DATAFLOW = 0, 1, 2, 3
CHOL_SCHED_LEFT_LOOKING, CHOL_SCHED_TOP_LOOKING = 4, 5
CHOL_FLAG_NOOP, CHOL_FLAG_PRIORITY, CHOL_FLAG_GRAPH, CHOL_FLAG_TEST_WITHHOLD, CHOL_FLAG_FP64_TC = 1, 2, 4, 8, 16
CHOL_FLAG_GMRES_IR = 32
CHOL_FLAG_FP64_SIMT = 64

PRECISIONS = {"fp64": CHOL_FP64, "fp32": CHOL_FP32, "tf32": CHOL_TF32, "bf16": CHOL_BF16, "fp16": CHOL_FP16}
SCHEDULES = {"auto": CHOL_SCHED_AUTO, "fork_join": CHOL_SCHED_FORK_JOIN,
             "fork_join_naive": CHOL_SCHED_FORK_JOIN_NAIVE, "dataflow": CHOL_SCHED_DATAFLOW,
             "left_looking": CHOL_SCHED_LEFT_LOOKING, "top_looking": CHOL_SCHED_TOP_LOOKING}

_i32, _i64, _dbl, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class chol_trace_rec(ctypes.Structure):
    _fields_ = [("type", _i32), ("I", _i32), ("K", _i32), ("J", _i32), ("sm", _i32), ("matrix", _i32),
                ("t_start", ctypes.c_uint64), ("t_end", ctypes.c_uint64)]


class chol_opts(ctypes.Structure):
    _fields_ = [("schedule", _i32), ("precision", _i32), ("nb", _i64), ("flags", _i32), ("max_iter", _i32),
                ("refine_tol", _dbl), ("timeout_s", _dbl), ("stream", _vp), ("num_ctas", _i32),
                ("tc_min_order", _i32), ("trace", _vp), ("trace_capacity", _i64)]


class chol_stats(ctypes.Structure):
    _fields_ = [("tasks", _i64 * 4), ("nb", _i64), ("schedule", _i32), ("launches", _i32),
                ("trace_records", _i64), ("device_ms", _dbl)]


class chol_request(ctypes.Structure):
    _fields_ = [("n", _i64), ("A", _vp), ("lda", _i64), ("factor_id", ctypes.c_uint64), ("B", _vp),
                ("ldb", _i64), ("X", _vp), ("ldx", _i64), ("nrhs", _i64), ("precision", _i32),
                ("reserved", _i32)]


class chol_result(ctypes.Structure):
    _fields_ = [("status", _i32), ("iters", _i32), ("info", _i64), ("berr", _dbl), ("latency_ms", _dbl),
                ("queue_ms", _dbl), ("reused_factor", _i32), ("slot", _i32)]


class chol_server_stats_t(ctypes.Structure):
    _fields_ = [("completed", _i64), ("failed", _i64), ("rejected", _i64), ("resident_factors", _i64),
                ("bytes_in_use", ctypes.c_size_t), ("budget", ctypes.c_size_t), ("p50_ms", _dbl),
                ("p99_ms", _dbl), ("mean_ms", _dbl), ("solves_per_s", _dbl), ("elapsed_s", _dbl)]


_P = ctypes.POINTER
# name -> (restype, argtypes), mirroring include/chol.h
SIGNATURES = {
    "chol_opts_init": (None, [_P(chol_opts)]),
    "chol_last_error": (ctypes.c_char_p, []),
    "chol_version": (ctypes.c_char_p, []),
    "chol_factor": (ctypes.c_int, [_i64, _i64, _vp, _i64]),
    "chol_last_info": (_i64, []),
    "chol_factor_ex": (ctypes.c_int, [_i64, _vp, _i64, _P(chol_opts), _P(_i64), _P(chol_stats)]),
    "chol_factor_host": (ctypes.c_int, [_i64, _vp, _i64, _P(chol_opts), _P(_i64), _P(chol_stats)]),
    "chol_solve": (ctypes.c_int, [_i64, _i64, _vp, _vp]),
    "chol_solve_ex": (ctypes.c_int, [_i64, _i64, _vp, _i64, _vp, _i64, _P(chol_opts)]),
    "chol_solve_noalloc": (ctypes.c_int, [_i64, _i64, _vp, _i64, _vp, _i64, _vp]),
    "chol_mixed_factor": (ctypes.c_int, [_i64, _vp, _i64, _P(chol_opts), _P(_vp), _P(_i64)]),
    "chol_mixed_solve": (ctypes.c_int, [_vp, _i64, _vp, _i64, _vp, _i64, _P(_i32), _P(_dbl)]),
    "chol_mixed_get_factor": (ctypes.c_int, [_vp, _vp, _i64]),
    "chol_factor_free": (None, [_vp]),
    "chol_mixed_last_stats": (ctypes.c_int, [_P(chol_stats)]),
    "chol_test_tc_update": (ctypes.c_int, [_i32, _i64, _vp, _i32, _i32, _vp, _i32]),
    "chol_test_ozaki_update": (ctypes.c_int, [_vp, _vp, _vp]),
    "chol_test_oz_residual": (ctypes.c_int, [_i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _i64]),
    "chol_test_device_memory": (ctypes.c_int, [_P(ctypes.c_uint64), _P(ctypes.c_uint64), _P(ctypes.c_uint64)]),
    "chol_batch_plan": (ctypes.c_int, [_i32, _P(_i64), _P(chol_opts), _P(_vp)]),
    "chol_batch_run": (ctypes.c_int, [_vp, _P(_vp), _P(_i64), _P(_vp), _P(_i64)]),
    "chol_batch_stats": (ctypes.c_int, [_vp, _P(chol_stats)]),
    "chol_batch_free": (None, [_vp]),
    "chol_autotune": (ctypes.c_int, [_i64, _i32, ctypes.c_char_p, _dbl, _P(chol_opts)]),
    "chol_default_nb": (_i64, [_i64, _i32]),
    "chol_server_create": (ctypes.c_int, [ctypes.c_size_t, _i32, _P(chol_opts), _P(_vp)]),
    "chol_server_submit": (ctypes.c_int, [_vp, _P(chol_request), _P(ctypes.c_uint64)]),
    "chol_server_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, _P(chol_result)]),
    "chol_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, _P(chol_result), _dbl]),
    "chol_server_release": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "chol_server_stats": (ctypes.c_int, [_vp, _P(chol_server_stats_t)]),
    "chol_server_destroy": (None, [_vp]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libchol.so (raises RuntimeError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libchol.so not found at {LIB_PATH}: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class CholError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().chol_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {status}: {msg}")


def _check(rc: int, where: str, ok=(CHOL_OK,)) -> int:
    if rc not in ok:
        raise CholError(rc, where)
    return rc


# --------------------------------------------------------------------- marshalling helpers
def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _ld(t) -> int:
    """Leading dimension of a column-major 2-D tensor (or n for a vector)."""
    if t.dim() == 1:
        return max(1, t.shape[0])
    if t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError("matrix must be column-major (stride(0) == 1); use colmajor()")
    return max(1, t.stride(1), t.shape[0])


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def colmajor(x, device="cuda", dtype=None):
    """Column-major torch copy of a 2-D numpy array or tensor on `device`."""
    import numpy as np
    import torch
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x))
    dtype = dtype or x.dtype
    out = torch.empty_strided(tuple(x.shape), (1, x.shape[0]) if x.dim() == 2 else (1,), dtype=dtype, device=device)
    out.copy_(x)
    return out


def opts(schedule="auto", precision="fp64", nb=0, flags=0, max_iter=30, refine_tol=1e-14, timeout_s=60.0,
         stream=None, num_ctas=0, trace=None, trace_capacity=0, tc_min_order=0) -> chol_opts:
    o = chol_opts()
    lib().chol_opts_init(ctypes.byref(o))
    o.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.nb = int(nb)
    o.flags = int(flags)
    o.max_iter = int(max_iter)
    o.refine_tol = float(refine_tol)
    o.timeout_s = float(timeout_s)
    o.stream = _stream() if stream is None else int(stream)
    o.num_ctas = int(num_ctas)
    o.tc_min_order = int(tc_min_order)
    o.trace = _ptr(trace) or None
    o.trace_capacity = int(trace_capacity)
    return o


# --------------------------------------------------------------------- entry points (same names)
def chol_version() -> str:
    return lib().chol_version().decode()


def chol_last_error() -> str:
    return lib().chol_last_error().decode()


def chol_default_nb(n: int, precision="fp64") -> int:
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return int(lib().chol_default_nb(int(n), p))


def chol_factor(n: int, nb: int, A, lda: int | None = None) -> int:
    """A = L L^T in place (FP64, dataflow).  Returns CHOL_OK, or raises; a
    matrix that is not SPD returns CHOL_ERR_NOT_SPD (info in chol_last_info)."""
    lda = _ld(A) if lda is None else lda
    rc = lib().chol_factor(int(n), int(nb), _ptr(A), int(lda))
    return _check(rc, "chol_factor", ok=(CHOL_OK, CHOL_ERR_NOT_SPD))


def chol_last_info() -> int:
    return int(lib().chol_last_info())


def chol_factor_ex(A, o: chol_opts | None = None, n: int | None = None, lda: int | None = None,
                   raise_on_error: bool = True):
    """Returns (status, info, stats)."""
    n = A.shape[0] if n is None else n
    lda = _ld(A) if lda is None else lda
    o = o or opts()
    info = _i64(0)
    st = chol_stats()
    rc = lib().chol_factor_ex(int(n), _ptr(A), int(lda), ctypes.byref(o), ctypes.byref(info), ctypes.byref(st))
    if raise_on_error:
        _check(rc, "chol_factor_ex")
    return rc, int(info.value), st


def chol_factor_host(A_host, o: chol_opts | None = None, n: int | None = None, lda: int | None = None):
    """Host-buffer factorization (A_host: column-major CPU tensor, ideally pinned)."""
    n = A_host.shape[0] if n is None else n
    lda = _ld(A_host) if lda is None else lda
    o = o or opts()
    info = _i64(0)
    st = chol_stats()
    rc = lib().chol_factor_host(int(n), _ptr(A_host), int(lda), ctypes.byref(o), ctypes.byref(info),
                                ctypes.byref(st))
    _check(rc, "chol_factor_host")
    return int(info.value), st


def chol_solve(n: int, nrhs: int, L, B) -> int:
    return _check(lib().chol_solve(int(n), int(nrhs), _ptr(L), _ptr(B)), "chol_solve")


def chol_solve_ex(L, B, o: chol_opts | None = None, n: int | None = None, nrhs: int | None = None,
                  raise_on_error: bool = True) -> int:
    n = L.shape[0] if n is None else n
    nrhs = (B.shape[1] if B.dim() == 2 else 1) if nrhs is None else nrhs
    o = o or opts()
    rc = lib().chol_solve_ex(int(n), int(nrhs), _ptr(L), _ld(L), _ptr(B), _ld(B), ctypes.byref(o))
    if raise_on_error:
        _check(rc, "chol_solve_ex")
    return rc


def chol_solve_noalloc(L, B, n: int | None = None, nrhs: int | None = None, stream=None) -> int:
    """Allocation-free FP64 solve (see include/chol.h): returns the status."""
    n = L.shape[0] if n is None else n
    nrhs = (B.shape[1] if B.dim() == 2 else 1) if nrhs is None else nrhs
    st = _stream() if stream is None else int(stream)
    return lib().chol_solve_noalloc(int(n), int(nrhs), _ptr(L), _ld(L), _ptr(B), _ld(B), st)


class MixedFactor:
    """Handle of chol_mixed_factor; frees the factor on close()/del."""

    def __init__(self, handle: int, info: int, A):
        self.h = handle
        self.info = info
        self._A = A  # the handle references A: keep it alive

    def solve(self, B, X=None, raise_on_error: bool = True):
        import torch
        nrhs = B.shape[1] if B.dim() == 2 else 1
        if X is None:
            X = torch.empty_strided(tuple(B.shape), B.stride(), dtype=torch.float64, device=B.device)
        it = _i32(0)
        be = _dbl(0.0)
        rc = lib().chol_mixed_solve(self.h, int(nrhs), _ptr(B), _ld(B), _ptr(X), _ld(X), ctypes.byref(it),
                                    ctypes.byref(be))
        if raise_on_error:
            _check(rc, "chol_mixed_solve", ok=(CHOL_OK, CHOL_ERR_NOT_CONVERGED))
        return rc, X, int(it.value), float(be.value)

    def factor(self, L=None):
        import torch
        n = self._A.shape[0]
        if L is None:
            L = torch.zeros((n, n), dtype=torch.float64, device=self._A.device).T
        _check(lib().chol_mixed_get_factor(self.h, _ptr(L), _ld(L)), "chol_mixed_get_factor")
        return L

    def close(self):
        if self.h:
            lib().chol_factor_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def chol_mixed_last_stats() -> chol_stats:
    st = chol_stats()
    _check(lib().chol_mixed_last_stats(ctypes.byref(st)), "chol_mixed_last_stats")
    return st


def chol_test_tc_update(precision, nb: int, ops, eA: int, eB: int, C, lower: bool = False) -> int:
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return lib().chol_test_tc_update(p, int(nb), _ptr(ops), int(eA), int(eB), _ptr(C), int(bool(lower)))


def chol_mixed_factor(A, o: chol_opts | None = None, raise_on_error: bool = True):
    o = o or opts(precision="tf32")
    h = _vp(None)
    info = _i64(0)
    rc = lib().chol_mixed_factor(int(A.shape[0]), _ptr(A), _ld(A), ctypes.byref(o), ctypes.byref(h),
                                 ctypes.byref(info))
    if raise_on_error:
        _check(rc, "chol_mixed_factor")
    return rc, (MixedFactor(h.value, int(info.value), A) if rc == CHOL_OK else None)


class BatchPlan:
    """Handle of chol_batch_plan (one persistent launch in a CUDA graph)."""

    def __init__(self, ns, o: chol_opts | None = None):
        self.ns = [int(x) for x in ns]
        arr = (_i64 * len(self.ns))(*self.ns)
        h = _vp(None)
        o = o or opts()
        _check(lib().chol_batch_plan(len(self.ns), arr, ctypes.byref(o), ctypes.byref(h)), "chol_batch_plan")
        self.h = h.value

    def run(self, As, Bs):
        """As: column-major CUDA tensors (overwritten by L), Bs: CUDA vectors
        (overwritten by the solutions).  Returns the list of info values."""
        k = len(self.ns)
        pa = (_vp * k)(*[_ptr(a) for a in As])
        lda = (_i64 * k)(*[_ld(a) for a in As])
        pb = (_vp * k)(*[_ptr(b) for b in Bs])
        info = (_i64 * k)()
        _check(lib().chol_batch_run(self.h, pa, lda, pb, info), "chol_batch_run")
        return list(info)

    def stats(self) -> chol_stats:
        st = chol_stats()
        _check(lib().chol_batch_stats(self.h, ctypes.byref(st)), "chol_batch_stats")
        return st

    def close(self):
        if self.h:
            lib().chol_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def chol_batch_plan(ns, o: chol_opts | None = None) -> BatchPlan:
    return BatchPlan(ns, o)


def chol_autotune(n: int, precision="fp64", cache_path: str | None = None, budget_s: float = 5.0) -> chol_opts:
    """Measured (nb, schedule) for order n; returns a chol_opts with them set."""
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o = chol_opts()
    _check(lib().chol_autotune(int(n), p, cache_path.encode() if cache_path else None, float(budget_s),
                               ctypes.byref(o)), "chol_autotune")
    return o


def _res_dict(r: chol_result) -> dict:
    return {f: getattr(r, f) for f, _ in chol_result._fields_}


class Server:
    """Handle of chol_server_create (continuous-batching solve server)."""

    def __init__(self, budget_bytes: int, slots: int = 4, o: chol_opts | None = None):
        h = _vp(None)
        o = o or opts()
        _check(lib().chol_server_create(int(budget_bytes), int(slots), ctypes.byref(o), ctypes.byref(h)),
               "chol_server_create")
        self.h = h.value

    def submit(self, B, X, A=None, factor_id: int = 0, precision="fp64", n: int | None = None) -> int:
        r = chol_request()
        r.n = int(n if n is not None else B.shape[0])
        r.A = _ptr(A) or None
        r.lda = _ld(A) if A is not None else 0
        r.factor_id = int(factor_id)
        r.B = _ptr(B)
        r.ldb = _ld(B)
        r.X = _ptr(X)
        r.ldx = _ld(X)
        r.nrhs = B.shape[1] if B.dim() == 2 else 1
        r.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        t = ctypes.c_uint64(0)
        _check(lib().chol_server_submit(self.h, ctypes.byref(r), ctypes.byref(t)), "chol_server_submit")
        return t.value

    def poll(self, ticket: int):
        r = chol_result()
        rc = lib().chol_server_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r))
        return rc, (_res_dict(r) if rc == CHOL_OK else None)

    def wait(self, ticket: int, timeout_s: float = 600.0) -> dict:
        r = chol_result()
        _check(lib().chol_server_wait(self.h, ctypes.c_uint64(ticket), ctypes.byref(r), float(timeout_s)),
               "chol_server_wait")
        return _res_dict(r)

    def release(self, factor_id: int) -> int:
        return lib().chol_server_release(self.h, ctypes.c_uint64(factor_id))

    def stats(self) -> dict:
        s = chol_server_stats_t()
        _check(lib().chol_server_stats(self.h, ctypes.byref(s)), "chol_server_stats")
        return {f: getattr(s, f) for f, _ in chol_server_stats_t._fields_}

    def close(self):
        if self.h:
            lib().chol_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
