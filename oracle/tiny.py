"""Second, independent restatement of Gaussian PLS on unpacked 0/1 arrays.

TEST INFRASTRUCTURE ONLY (same import rule as the rest of ``oracle/``). Pure
Python + numpy bool rows, written separately from ``gf2_oracle.c`` so that a
slip in either one shows up as a disagreement. Intended for matrices up to
about 64 x 64.

It also provides the decomposition helpers that turn the in-place result into
explicit factors, and the product P.L.S used to reconstruct A.
"""
from __future__ import annotations

import numpy as np


def gauss_pls(M: np.ndarray):
    """Gaussian PLS of a 0/1 matrix (appendix algorithm), returns (A', P, Q, r)."""
    A = np.array(M, dtype=bool, copy=True)
    m, n = A.shape
    P = list(range(m))
    Q = list(range(n))
    r = 0
    c = 0
    while r < m and c < n:
        hit = None
        for j in range(c, n):
            rows = np.nonzero(A[r:, j])[0]
            if rows.size:
                hit = (r + int(rows[0]), j)
                break
        if hit is None:
            break
        i, j = hit
        P[r], Q[r] = i, j
        A[[r, i]] = A[[i, r]]
        for l in range(r + 1, m):
            if A[l, j]:
                A[l, j + 1:] ^= A[r, j + 1:]
        r += 1
        c = j + 1
    for i in range(r, m):
        P[i] = i
    for i in range(r, n):
        Q[i] = i
    for j in range(r):
        q = Q[j]
        if q != j:
            tmp = A[j:, j].copy()
            A[j:, j] = A[j:, q]
            A[j:, q] = tmp
    return A.astype(np.uint8), np.array(P, dtype=np.int64), np.array(Q, dtype=np.int64), r


def factors(Ain: np.ndarray, P: np.ndarray, Q: np.ndarray, r: int):
    """Explicit (L, S) from the compressed in-place PLS result.

    Row i < r of the result is [L_i (cols < i) | 1 at i | 0 up to Q[i] |
    S_i right of Q[i] in original positions]; rows >= r hold L in cols < r.
    L is m x r unit lower trapezoidal, S is r x n with its leading 1 at Q[i].
    """
    A = np.asarray(Ain, dtype=np.uint8)
    m, n = A.shape
    L = np.zeros((m, r), dtype=np.uint8)
    S = np.zeros((r, n), dtype=np.uint8)
    for i in range(m):
        w = min(i, r)
        L[i, :w] = A[i, :w]
        if i < r:
            L[i, i] = 1
    for i in range(r):
        q = int(Q[i])
        S[i, q] = 1
        S[i, q + 1:] = A[i, q + 1:]
    return L, S


def apply_swaps_rows(M: np.ndarray, P: np.ndarray, upto: int, reverse: bool) -> np.ndarray:
    """Apply the transpositions i <-> P[i] (i < upto) to the rows of M."""
    M = np.array(M, copy=True)
    order = range(upto - 1, -1, -1) if reverse else range(upto)
    for i in order:
        p = int(P[i])
        if p != i:
            M[[i, p]] = M[[p, i]]
    return M


def reconstruct(Ain: np.ndarray, P: np.ndarray, Q: np.ndarray, r: int) -> np.ndarray:
    """A = P.L.S : apply the swaps i = r-1 .. 0 to the rows of L.S."""
    L, S = factors(Ain, P, Q, r)
    LS = (L.astype(np.int64) @ S.astype(np.int64)) % 2
    return apply_swaps_rows(LS.astype(np.uint8), P, r, reverse=True)
