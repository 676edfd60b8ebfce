"""FP64 reference GEMM (Section 3) -- TEST INFRASTRUCTURE ONLY.

Thin ctypes front end over ``gemm_ref.c`` (plain C triple loop).  Inputs are
converted exactly to float64 (every float32 and bfloat16 value is a float64
value), so the only rounding is FP64's own.

Pinned by ``tests/test_oracle_gemm.py``: identity and permutation products,
rank-1 and all-ones closed forms, a closed-form polynomial product that is
asymmetric in every index, small-integer exactness, and the componentwise
scale on non-negative data.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_gemm.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gemm_ref.c with gcc (-O2, OpenMP).  Returns the .so path."""
    src = os.path.join(_HERE, "gemm_ref.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dbl, ptr = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.oracle_gemm.argtypes = [ctypes.c_int, ctypes.c_int, i64, i64, i64, i64, dbl,
                                        ptr, i64, i64, ptr, i64, i64, dbl, ptr, i64, i64,
                                        ptr, ptr, ctypes.c_int]
            lib.oracle_gemm.restype = None
            lib.oracle_gemm_entries.argtypes = [ctypes.c_int, ctypes.c_int, i64, dbl,
                                                ptr, i64, i64, ptr, i64, i64, dbl, ptr, i64, i64,
                                                i64, ptr, ptr, ptr, ctypes.c_int]
            lib.oracle_gemm_entries.restype = None
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _as3(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x)
    if x.ndim == 2:
        x = x[None]
    return np.ascontiguousarray(x, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def gemm(transA: str, transB: str, M: int, N: int, K: int, alpha: float, A, B, beta: float = 0.0,
         C0=None, nthreads: int = 1):
    """C = alpha*op(A)*op(B) + beta*C0 and den = |alpha||op(A)||op(B)| + |beta||C0|.

    A, B, C0 are (batch, rows, ld) or (rows, ld) arrays as stored (row-major,
    ld = last dimension); returns (C, den), each float64 (batch, M, N).
    """
    lib = _load()
    A3, B3 = _as3(A), _as3(B)
    batch = A3.shape[0]
    assert B3.shape[0] == batch
    ta, tb = int(transA == "T"), int(transB == "T")
    ar, ac = (K, M) if ta else (M, K)
    br, bc = (N, K) if tb else (K, N)
    assert A3.shape[1] >= ar and A3.shape[2] >= ac, (A3.shape, ar, ac)
    assert B3.shape[1] >= br and B3.shape[2] >= bc, (B3.shape, br, bc)
    if beta != 0.0:
        C3 = _as3(C0)
        assert C3.shape[0] == batch and C3.shape[1] >= M and C3.shape[2] >= N
        ldc, sc = C3.shape[2], C3.shape[1] * C3.shape[2]
    else:
        C3, ldc, sc = None, 0, 0
    C = np.empty((batch, M, N), np.float64)
    den = np.empty((batch, M, N), np.float64)
    if M and N and batch:
        lib.oracle_gemm(ta, tb, M, N, K, batch, float(alpha),
                        _ptr(A3), A3.shape[2], A3.shape[1] * A3.shape[2],
                        _ptr(B3), B3.shape[2], B3.shape[1] * B3.shape[2], float(beta),
                        _ptr(C3), ldc, sc, _ptr(C), _ptr(den), int(nthreads))
    return C, den


def gemm_entries(transA: str, transB: str, M: int, N: int, K: int, alpha: float, A, B, beta: float,
                 C0, pos: np.ndarray, nthreads: int = 1):
    """Entries (b, i, j) listed in ``pos`` (n x 3 int64) of the same product; returns (C, den) of length n."""
    lib = _load()
    A3, B3 = _as3(A), _as3(B)
    pos = np.ascontiguousarray(pos, dtype=np.int64)
    assert pos.ndim == 2 and pos.shape[1] == 3
    if len(pos):
        assert pos[:, 1].max() < M and pos[:, 2].max() < N and pos[:, 0].max() < A3.shape[0]
    if beta != 0.0:
        C3 = _as3(C0)
        ldc, sc = C3.shape[2], C3.shape[1] * C3.shape[2]
    else:
        C3, ldc, sc = None, 0, 0
    n = pos.shape[0]
    C = np.empty(n, np.float64)
    den = np.empty(n, np.float64)
    if n:
        lib.oracle_gemm_entries(int(transA == "T"), int(transB == "T"), K, float(alpha),
                                _ptr(A3), A3.shape[2], A3.shape[1] * A3.shape[2],
                                _ptr(B3), B3.shape[2], B3.shape[1] * B3.shape[2], float(beta),
                                _ptr(C3), ldc, sc, n, _ptr(pos), _ptr(C), _ptr(den), int(nthreads))
    return C, den


def error_ratio(C, C_ref, den) -> float:
    """max over entries of |C - C_ref| / den.  Where den == 0 the exact result
    is 0 and any nonzero C gives +inf; a NaN anywhere gives +inf."""
    C = np.asarray(C, np.float64)
    C_ref = np.asarray(C_ref, np.float64)
    den = np.asarray(den, np.float64)
    if C.size == 0:
        return 0.0
    diff = np.abs(C - C_ref)
    if not np.all(np.isfinite(diff)):
        return float("inf")
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(den > 0, diff / np.where(den > 0, den, 1.0), np.where(diff > 0, np.inf, 0.0))
    return float(r.max())
