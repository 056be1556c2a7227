"""CPU oracle for GF(2) PLS / rank / RREF / product -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package. It shares no code with the CUDA path.

``liboracle_gf2.so`` is compiled from ``gf2_oracle.c`` with the host C
compiler (``build()``). Functions take packed numpy uint64 arrays of shape
(m, stride) (column j = bit j&63 of word j>>6) and work on copies unless the
name says ``_inplace``.

Pins (what fixes each function independently of itself) live in
``tests/test_oracle_pins.py``; every oracle function is pinned there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf2_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_gf2.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain -O2, no vectorisation flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_HERE, "liboracle_gf2_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str:
    """The same source compiled with OpenMP (only gf2o_pls_omp differs): the all-cores timing variant."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def pls_omp(A: np.ndarray, m: int, n: int):
    """Gaussian PLS with OpenMP threads over the rows of each step (timing variant; same result)."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            build_omp()
            lib = ctypes.CDLL(_LIB_OMP)
            lib.gf2o_pls_omp.restype = _i64
            lib.gf2o_pls_omp.argtypes = [_p, _i64, _i64, _i64, _p, _p]
            _lib_omp = lib
    A = _mat(A).copy()
    P = np.zeros(max(m, 1), dtype=np.int64)
    Q = np.zeros(max(n, 1), dtype=np.int64)
    r = _lib_omp.gf2o_pls_omp(_ptr(A), m, n, A.shape[1], _ptr(P), _ptr(Q))
    return A, P[:m], Q[:n], int(r)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.gf2o_pls.restype = _i64
            lib.gf2o_pls.argtypes = [_p, _i64, _i64, _i64, _p, _p]
            lib.gf2o_rref.restype = _i64
            lib.gf2o_rref.argtypes = [_p, _i64, _i64, _i64, _p]
            lib.gf2o_mul.restype = None
            lib.gf2o_mul.argtypes = [_p, _i64, _p, _i64, _p, _i64, _i64, _i64, _i64, ctypes.c_int]
            lib.gf2o_pls_mmpf.restype = _i64
            lib.gf2o_pls_mmpf.argtypes = [_p, _i64, _i64, _i64, _p, _p, ctypes.c_int]
            lib.gf2o_pls_rec.restype = _i64
            lib.gf2o_pls_rec.argtypes = [_p, _i64, _i64, _i64, _p, _p, _i64, ctypes.c_int, ctypes.c_int]
            lib.gf2o_m4ri.restype = _i64
            lib.gf2o_m4ri.argtypes = [_p, _i64, _i64, _i64, ctypes.c_int, _p]
            lib.gf2o_make_table.restype = None
            lib.gf2o_make_table.argtypes = [_p, _i64, _i64, _i64, ctypes.c_int, _i64, ctypes.c_int, _p, _i64, _p]
            lib.gf2o_add_rows_from_table.restype = None
            lib.gf2o_add_rows_from_table.argtypes = [_p, _i64, _i64, _i64, _i64, _i64, ctypes.c_int, _p, _i64, _p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _mat(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.uint64)
    assert A.ndim == 2
    return A


def pls(A: np.ndarray, m: int, n: int):
    """Gaussian PLS. Returns (in-place result, P, Q, r) with P len m, Q len n."""
    A = _mat(A).copy()
    P = np.zeros(max(m, 1), dtype=np.int64)
    Q = np.zeros(max(n, 1), dtype=np.int64)
    r = _load().gf2o_pls(_ptr(A), m, n, A.shape[1], _ptr(P), _ptr(Q))
    return A, P[:m], Q[:n], int(r)


def rref(A: np.ndarray, m: int, n: int):
    """Gauss-Jordan RREF. Returns (R, pivots (len r), r)."""
    A = _mat(A).copy()
    piv = np.zeros(max(min(m, n), 1), dtype=np.int64)
    r = _load().gf2o_rref(_ptr(A), m, n, A.shape[1], _ptr(piv))
    return A, piv[:r], int(r)


def rank(A: np.ndarray, m: int, n: int) -> int:
    return rref(A, m, n)[2]


def mul(A: np.ndarray, B: np.ndarray, m: int, k: int, n: int, C: np.ndarray | None = None,
        stride: int | None = None) -> np.ndarray:
    """C = A.B (C is None) or C + A.B over GF(2); returns a new array."""
    A = _mat(A)
    B = _mat(B)
    if C is None:
        s = stride if stride is not None else max(16, ((n + 63) // 64 + 15) // 16 * 16)
        out = np.zeros((m, s), dtype=np.uint64)
        acc = 0
    else:
        out = _mat(C).copy()
        acc = 1
    _load().gf2o_mul(_ptr(out), out.shape[1], _ptr(A), A.shape[1], _ptr(B), B.shape[1], m, k, n, acc)
    return out


def pls_mmpf(A: np.ndarray, m: int, n: int, k: int):
    """Literal Algorithm MMPF (PlsSubmatrix, MakeTable1, AddRowsFromTable)."""
    A = _mat(A).copy()
    P = np.zeros(max(m, 1), dtype=np.int64)
    Q = np.zeros(max(n, 1), dtype=np.int64)
    r = _load().gf2o_pls_mmpf(_ptr(A), m, n, A.shape[1], _ptr(P), _ptr(Q), k)
    assert r >= 0
    return A, P[:m], Q[:n], int(r)


def pls_rec(A: np.ndarray, m: int, n: int, cutoff: int, k: int, split_words: bool = False):
    """Literal recursive Algorithm PLS with an MMPF base case at n <= cutoff."""
    A = _mat(A).copy()
    P = np.zeros(max(m, 1), dtype=np.int64)
    Q = np.zeros(max(n, 1), dtype=np.int64)
    r = _load().gf2o_pls_rec(_ptr(A), m, n, A.shape[1], _ptr(P), _ptr(Q), cutoff, k, int(split_words))
    assert r >= 0
    return A, P[:m], Q[:n], int(r)


def m4ri(A: np.ndarray, m: int, n: int, k: int):
    """Literal Algorithm M4RI (GaussSubmatrix, MakeTable, AddRowsFromTable above and below).
    Returns (R, pivots (len r), r) like rref()."""
    A = _mat(A).copy()
    piv = np.zeros(max(min(m, n), 1), dtype=np.int64)
    r = _load().gf2o_m4ri(_ptr(A), m, n, A.shape[1], k, _ptr(piv))
    assert r >= 0
    return A, piv[:r], int(r)


def make_table(A: np.ndarray, n: int, r: int, k: int, c: int, fix: bool):
    """MakeTable (fix=False) / MakeTable1 (fix=True) over rows r..r+k-1."""
    A = _mat(A)
    ts = (n + 63) // 64 + 1
    T = np.zeros((1 << k, ts), dtype=np.uint64)
    L = np.zeros(1 << k, dtype=np.int64)
    _load().gf2o_make_table(_ptr(A), A.shape[1], n, r, k, c, int(fix), _ptr(T), ts, _ptr(L))
    return T, L


def add_rows_from_table(A: np.ndarray, n: int, rs: int, re: int, c: int, k: int, T: np.ndarray,
                        L: np.ndarray) -> np.ndarray:
    A = _mat(A).copy()
    T = _mat(T)
    L = np.ascontiguousarray(L, dtype=np.int64)
    _load().gf2o_add_rows_from_table(_ptr(A), A.shape[1], n, rs, re, c, k, _ptr(T), T.shape[1], _ptr(L))
    return A
