"""CPU oracle for the generalized sparse contraction path.  TEST INFRASTRUCTURE.

Only the tests, the package's smoke check and the benchmark's CPU-baseline arm
load this module.  It never imports the CUDA package and the CUDA package never
imports it.  The arithmetic lives in ``stc_oracle.c`` (plain C, fp64 where the
algebra is floating point, OpenMP across independent rows or sources); this
file compiles it with gcc on first use and wraps it with ctypes.

Algebra ids:  PT_F32=0 (+,x) fp32 operands, fp64 result;  PT_F64=1;
MP_I32=2 (min,+) int32;  MP_F32=3 (min,+) fp32;  BOOL=4 (or,and);
MULTPATH=5 (distance, multiplicity) monoid.

Parity is pinned for every function here by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (brute force, closed forms, scipy/networkx).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from workloads import MULTPATH_DTYPE, Csr

PT_F32, PT_F64, MP_I32, MP_F32, BOOL, MULTPATH = range(6)
TROP_I32_ID = (2 ** 31 - 1) // 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stc_oracle.c")
_LIB = os.path.join(_HERE, "libstc_oracle.so")
_lock = threading.Lock()
_lib = None

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_spgemm_count.argtypes = [_i64, _i64, _p, _p, _p, _p, _p, _i64, _p]
            L.orc_spgemm_fill.argtypes = [ctypes.c_int, _i64, _i64, _p, _p, _p, _p, _p, _p,
                                          _p, _i64, _p, _p, _p, _p]
            L.orc_spmm.argtypes = [ctypes.c_int, _i64, _p, _p, _p, _p, _i64, _i32, _p, _i64,
                                   ctypes.c_int]
            L.orc_bellman_ford.argtypes = [ctypes.c_int, _i64, _p, _p, _p, _i32, _p, _p]
            L.orc_bellman_ford.restype = _i64
            L.orc_dijkstra.argtypes = [ctypes.c_int, _i64, _p, _p, _p, _i32, _p]
            L.orc_floyd_warshall_i32.argtypes = [_i64, _p]
            L.orc_brandes.argtypes = [_i64, _p, _p, _p, ctypes.c_int, _p, _i64, _p]
            L.orc_sssp_counts.argtypes = [_i64, _p, _p, _p, ctypes.c_int, _i32, _p, _p]
            L.orc_splitmix64.argtypes = [ctypes.c_uint64]
            L.orc_splitmix64.restype = ctypes.c_uint64
            L.orc_row_features.argtypes = [_p, _p, _p, _p, _p, _i64, _p]
            L.orc_mlp_num_weights.restype = ctypes.c_int
            L.orc_mlp_forward.argtypes = [_p, _p, _i64, _p]
            L.orc_mlp_grad.argtypes = [_p, _p, _p, _i64, _p, _p]
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    lib().orc_set_threads(ctypes.c_int(n))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def value_dtype(alg: int, operand: str = "A"):
    """Element type of A / B(X) / C for an algebra.  C of (+,x) is fp64 here."""
    if alg == PT_F32:
        return np.float64 if operand == "C" else np.float32
    if alg == PT_F64:
        return np.float64
    if alg == MP_I32:
        return np.int32
    if alg == MP_F32:
        return np.float32
    if alg == BOOL:
        return np.uint8
    if alg == MULTPATH:
        return np.int32 if operand == "A" else MULTPATH_DTYPE
    raise ValueError(alg)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def spgemm_count(A: Csr, B: Csr, rows=None) -> np.ndarray:
    assert A.ncols == B.nrows
    rows_a = None if rows is None else _c(rows, np.int64)
    nsel = A.nrows if rows_a is None else rows_a.size
    counts = np.zeros(nsel, dtype=np.int64)
    lib().orc_spgemm_count(A.nrows, B.ncols, _ptr(_c(A.rowptr, np.int64)), _ptr(_c(A.col, np.int32)),
                           _ptr(_c(B.rowptr, np.int64)), _ptr(_c(B.col, np.int32)),
                           _ptr(rows_a), nsel, _ptr(counts))
    return counts


def spgemm(alg: int, A: Csr, B: Csr, rows=None, want_abs: bool = False):
    """C = A (x) B for all rows (rows=None) or the listed rows, in that order.

    Returns (rowptr, col, val, abs) over the selected rows; abs is the fp64 sum
    of |a*b| per entry for the (+,x) algebras (None otherwise or if not wanted).
    """
    assert A.ncols == B.nrows
    rows_a = None if rows is None else _c(rows, np.int64)
    counts = spgemm_count(A, B, rows_a)
    ptr = np.zeros(counts.size + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    nnz = int(ptr[-1])
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=value_dtype(alg, "C"))
    ab = np.zeros(nnz, dtype=np.float64) if (want_abs and alg in (PT_F32, PT_F64)) else None
    av = _c(A.val, value_dtype(alg, "A"))
    bv = _c(B.val, value_dtype(alg, "B"))
    lib().orc_spgemm_fill(alg, A.nrows, B.ncols, _ptr(_c(A.rowptr, np.int64)), _ptr(_c(A.col, np.int32)),
                          _ptr(av), _ptr(_c(B.rowptr, np.int64)), _ptr(_c(B.col, np.int32)), _ptr(bv),
                          _ptr(rows_a), counts.size, _ptr(ptr), _ptr(col), _ptr(val), _ptr(ab))
    return ptr, col, val, ab


def spmm(alg: int, A: Csr, X: np.ndarray, Y0: np.ndarray = None) -> np.ndarray:
    """Y = A (x) X (or Y0 (+) A (x) X) with X dense [A.ncols, ncol] (or a vector)."""
    vec = X.ndim == 1
    X2 = X.reshape(X.shape[0], -1)
    xd = value_dtype(alg, "B")
    X2 = _c(X2, xd)
    ncol = X2.shape[1]
    Y = np.zeros((A.nrows, ncol), dtype=xd) if Y0 is None else _c(Y0.reshape(A.nrows, ncol), xd).copy()
    av = _c(A.val, value_dtype(alg, "A"))
    lib().orc_spmm(alg, A.nrows, _ptr(_c(A.rowptr, np.int64)), _ptr(_c(A.col, np.int32)), _ptr(av),
                   _ptr(X2), ncol, ncol, _ptr(Y), ncol, 0 if Y0 is None else 1)
    return Y.reshape(-1) if vec else Y


def spmv(alg: int, A: Csr, x: np.ndarray, y0: np.ndarray = None) -> np.ndarray:
    return spmm(alg, A, x.reshape(-1), y0)


def bellman_ford(alg: int, G: Csr, source: int, with_relaxations: bool = False):
    """Returns (dist, rounds); rounds == -1 signals a reachable negative cycle.
    With with_relaxations, returns (dist, rounds, number of edge relaxations)."""
    d = np.zeros(G.nrows, dtype=np.int32 if alg == MP_I32 else np.float32)
    w = _c(G.val, d.dtype)
    relax = np.zeros(1, dtype=np.int64)
    r = lib().orc_bellman_ford(alg, G.nrows, _ptr(_c(G.rowptr, np.int64)), _ptr(_c(G.col, np.int32)),
                               _ptr(w), int(source), _ptr(d), _ptr(relax))
    if with_relaxations:
        return d, int(r), int(relax[0])
    return d, int(r)


def dijkstra(alg: int, G: Csr, source: int) -> np.ndarray:
    d = np.zeros(G.nrows, dtype=np.int32 if alg == MP_I32 else np.float32)
    w = _c(G.val, d.dtype)
    lib().orc_dijkstra(alg, G.nrows, _ptr(_c(G.rowptr, np.int64)), _ptr(_c(G.col, np.int32)),
                       _ptr(w), int(source), _ptr(d))
    return d


def floyd_warshall_i32(D: np.ndarray) -> np.ndarray:
    D = _c(D, np.int32).copy()
    lib().orc_floyd_warshall_i32(D.shape[0], _ptr(D))
    return D


def brandes(G: Csr, sources, weighted: bool) -> np.ndarray:
    src = _c(sources, np.int32)
    bc = np.zeros(G.nrows, dtype=np.float64)
    w = _c(G.val, np.int32) if weighted else np.zeros(1, np.int32)
    lib().orc_brandes(G.nrows, _ptr(_c(G.rowptr, np.int64)), _ptr(_c(G.col, np.int32)), _ptr(w),
                      1 if weighted else 0, _ptr(src), src.size, _ptr(bc))
    return bc


def sssp_counts(G: Csr, source: int, weighted: bool):
    d = np.zeros(G.nrows, dtype=np.int32)
    s = np.zeros(G.nrows, dtype=np.float64)
    w = _c(G.val, np.int32) if weighted else np.zeros(1, np.int32)
    lib().orc_sssp_counts(G.nrows, _ptr(_c(G.rowptr, np.int64)), _ptr(_c(G.col, np.int32)), _ptr(w),
                          1 if weighted else 0, int(source), _ptr(d), _ptr(s))
    return d, s


# ----------------------------------------------------------------- learned row sizing

NFEAT = 67
NHID = 64


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(x)))


def row_features(A: Csr, B: Csr, rows=None) -> np.ndarray:
    """fp64 features [len(rows), 67] of the output rows of A B (see stc_oracle.c)."""
    rows = np.arange(A.nrows, dtype=np.int64) if rows is None else _c(rows, np.int64)
    f = np.zeros((rows.size, NFEAT), dtype=np.float64)
    lib().orc_row_features(_ptr(_c(A.rowptr, np.int64)), _ptr(_c(A.col, np.int32)),
                           _ptr(_c(B.rowptr, np.int64)), _ptr(_c(B.col, np.int32)), _ptr(rows),
                           rows.size, _ptr(f))
    return f


def mlp_num_weights() -> int:
    return int(lib().orc_mlp_num_weights())


def mlp_forward(w: np.ndarray, x: np.ndarray) -> np.ndarray:
    x = _c(x, np.float64)
    y = np.zeros(x.shape[0], dtype=np.float64)
    lib().orc_mlp_forward(_ptr(_c(w, np.float64)), _ptr(x), x.shape[0], _ptr(y))
    return y


def mlp_grad(w: np.ndarray, x: np.ndarray, t: np.ndarray):
    """(gradient of the mean squared error w.r.t. the weights, loss), fp64."""
    x = _c(x, np.float64)
    g = np.zeros(mlp_num_weights(), dtype=np.float64)
    loss = np.zeros(1, dtype=np.float64)
    lib().orc_mlp_grad(_ptr(_c(w, np.float64)), _ptr(x), _ptr(_c(t, np.float64)), x.shape[0], _ptr(g),
                       _ptr(loss))
    return g, float(loss[0])
