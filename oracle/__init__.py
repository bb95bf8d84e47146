"""CPU oracle for the tiled right-looking Cholesky factorization (Section 3.1,
Fig. 1) and the SPD solve built on it.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may import this package.  The CUDA library never
imports, links or calls it, and it shares no code with the library: the C
sources here (``oracle.c``) are compiled with gcc into ``liboracle.so`` and
called through ctypes.

Every wrapper takes and returns numpy float64 arrays in Fortran (column-major)
order, the layout of the C functions (see ``oracle.h``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

# -ffp-contract=off: every + - * is rounded on its own (no FMA contraction), on
# x86_64 and aarch64 alike, so the oracle's arithmetic is exactly as written.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math"]


def build(src: str = _SRC, out: str = _LIB, extra: list[str] | None = None) -> str:
    """Compile ``src`` (default: oracle.c) into the shared library ``out``."""
    cmd = ["gcc", *CFLAGS, *(extra or []), "-I", _HERE, src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def _stale() -> bool:
    if not os.path.exists(_LIB):
        return True
    t = os.path.getmtime(_LIB)
    return any(os.path.getmtime(p) > t for p in (_SRC, _HDR))


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load (building first if needed) an oracle library and declare its ABI."""
    global _lib
    if path is None:
        if _lib is not None:
            return _lib
        if _stale():
            build()
        path = _LIB
    lib = ctypes.CDLL(path)
    i64, dp, i32p = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    sig = {
        "oracle_potrf_unblocked": (i64, [i64, dp, i64]),
        "oracle_potrf_tile": (i64, [i64, dp]),
        "oracle_trsm_tile": (None, [i64, dp, dp]),
        "oracle_syrk_tile": (None, [i64, dp, dp]),
        "oracle_gemm_tile": (None, [i64, dp, dp, dp]),
        "oracle_potrf_tiled": (i64, [i64, i64, dp, i64, i64p, i32p]),
        "oracle_potrf_tiled_tasks": (i64, [i64, i64, dp, i64, ctypes.c_int]),
        "oracle_max_threads": (ctypes.c_int, []),
        "oracle_potrs": (None, [i64, i64, dp, i64, dp, i64]),
        "oracle_residual_fro": (ctypes.c_double, [i64, dp, i64, dp, i64]),
        "oracle_residual_probe": (ctypes.c_double, [i64, dp, i64, dp, i64, i64, dp]),
        "oracle_backward_error": (ctypes.c_double, [i64, i64, dp, i64, dp, i64, dp, i64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path == _LIB:
        _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, copy: bool = True) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    return np.array(a, dtype=np.float64, order="F", copy=True) if copy else np.asfortranarray(a)


def potrf_unblocked(A, lib=None):
    """Return (L, info): L = lower factor of A (upper triangle of A kept as given)."""
    lib = lib or load()
    W = _f64(A)
    n = W.shape[0]
    info = lib.oracle_potrf_unblocked(n, _dp(W), max(1, n))
    return W, int(info)


def potrf_tiled(A, nb, lib=None, with_log: bool = False):
    """Fig. 1 on tiles of order nb.  Returns (L, info, counts[, log])."""
    lib = lib or load()
    W = _f64(A)
    n = W.shape[0]
    counts = np.zeros(4, dtype=np.int64)
    m = -(-n // nb) if n > 0 else 0
    ntask = m * (m + 1) * (m + 2) // 6
    log = np.zeros(4 * max(ntask, 1), dtype=np.int32) if with_log else None
    info = lib.oracle_potrf_tiled(
        n, nb, _dp(W), max(1, n), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        log.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if log is not None else None,
    )
    if with_log:
        return W, int(info), counts, log.reshape(-1, 4)[: int(counts.sum())]
    return W, int(info), counts


def potrf_tiled_tasks(A, nb, nthreads=0, lib=None):
    """OpenMP-task version of Fig. 1 (the timed CPU baseline).  Returns (L, info)."""
    lib = lib or load()
    W = _f64(A)
    n = W.shape[0]
    info = lib.oracle_potrf_tiled_tasks(n, nb, _dp(W), max(1, n), int(nthreads))
    return W, int(info)


def max_threads(lib=None) -> int:
    return int((lib or load()).oracle_max_threads())


def tile_op(op: str, *tiles, lib=None):
    """Apply one tile operation to row-major nb x nb tiles; returns the updated
    output tile (a copy).  op in {'potrf', 'trsm', 'syrk', 'gemm'}; for potrf
    the result is (tile, info)."""
    lib = lib or load()
    ts = [np.ascontiguousarray(np.asarray(t, dtype=np.float64)).copy() for t in tiles]
    nb = ts[0].shape[0]
    if op == "potrf":
        info = lib.oracle_potrf_tile(nb, _dp(ts[0]))
        return ts[0], int(info)
    if op == "trsm":
        lib.oracle_trsm_tile(nb, _dp(ts[0]), _dp(ts[1]))
        return ts[1]
    if op == "syrk":
        lib.oracle_syrk_tile(nb, _dp(ts[0]), _dp(ts[1]))
        return ts[1]
    if op == "gemm":
        lib.oracle_gemm_tile(nb, _dp(ts[0]), _dp(ts[1]), _dp(ts[2]))
        return ts[2]
    raise ValueError(op)


def potrs(L, B, lib=None):
    """Solve (L L^T) X = B; returns X."""
    lib = lib or load()
    Lf = _f64(L, copy=False)
    X = _f64(B)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    n, nrhs = X.shape
    lib.oracle_potrs(n, nrhs, _dp(Lf), max(1, Lf.shape[0]), _dp(X), max(1, n))
    return X


def residual_fro(A, L, lib=None) -> float:
    lib = lib or load()
    Af, Lf = _f64(A, copy=False), _f64(L, copy=False)
    n = Af.shape[0]
    return float(lib.oracle_residual_fro(n, _dp(Af), max(1, n), _dp(Lf), max(1, Lf.shape[0])))


def residual_probe(A, L, X, lib=None) -> float:
    lib = lib or load()
    Af, Lf, Xf = _f64(A, copy=False), _f64(L, copy=False), _f64(X, copy=False)
    if Xf.ndim == 1:
        Xf = Xf.reshape(-1, 1, order="F")
    n = Af.shape[0]
    return float(lib.oracle_residual_probe(n, _dp(Af), max(1, n), _dp(Lf), max(1, Lf.shape[0]),
                                           Xf.shape[1], _dp(Xf)))


def backward_error(A, X, B, lib=None) -> float:
    lib = lib or load()
    Af, Xf, Bf = _f64(A, copy=False), _f64(X, copy=False), _f64(B, copy=False)
    if Xf.ndim == 1:
        Xf = Xf.reshape(-1, 1, order="F")
        Bf = Bf.reshape(-1, 1, order="F")
    n = Af.shape[0]
    return float(lib.oracle_backward_error(n, Xf.shape[1], _dp(Af), max(1, n), _dp(Xf), max(1, n),
                                           _dp(Bf), max(1, n)))
