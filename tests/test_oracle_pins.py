"""Pins for the CPU oracle: values and facts fixed by the paper and by the
mathematics, not by the oracle itself (CPU only).

* Worked examples of the paper (golden files): MakeTable / AddRowsFromTable
  (Sec. 3.1, Figure "M4RI Idea"), MakeTable1's multipliers (Sec. 4.1).
* Rank: brute-force span size on small matrices, exhaustive counts over all
  3x3 / 4x4 / 2x8 / 3x5 / 5x3 matrices against the closed form
  prod_{i<r} (2^m-2^i)(2^n-2^i)/(2^r-2^i).
* PLS: reconstruction A = P.L.S, shape of L and S (Proposition "PLS
  decomposition"), agreement with an independent restatement, and the
  equivalence of Gaussian PLS, MMPF and recursive PLS claimed by the paper.
* RREF: uniqueness under left multiplication by invertible matrices,
  idempotence, structure (Definition "Reduced Row Echelon Form"), row space.
* Product: integer matrix product mod 2.
"""
from __future__ import annotations

import itertools
import os

import numpy as np
import pytest

import oracle
import oracle.tiny as tiny
from paper_1006_1744_gb300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = np.array([int(v) for v in vals], dtype=np.uint8)
    return rows


def span_rank(U: np.ndarray) -> int:
    """Rank by brute force: |row space| = 2^r, enumerating all combinations."""
    m, n = U.shape
    vecs = set()
    ints = [int("".join(str(int(b)) for b in row) or "0", 2) for row in U]
    for mask in range(1 << m):
        acc = 0
        for i in range(m):
            if mask >> i & 1:
                acc ^= ints[i]
        vecs.add(acc)
    return len(vecs).bit_length() - 1


def count_rank(m: int, n: int, r: int) -> int:
    num = 1
    den = 1
    for i in range(r):
        num *= (2 ** m - 2 ** i) * (2 ** n - 2 ** i)
        den *= 2 ** r - 2 ** i
    return num // den


def all_matrices(m, n):
    for bits in range(1 << (m * n)):
        U = np.array([(bits >> t) & 1 for t in range(m * n)], dtype=np.uint8).reshape(m, n)
        yield U


# ----------------------------------------------------------------------------
# worked examples of the paper
# ----------------------------------------------------------------------------

def test_fig1_maketable_golden():
    g = _golden("fig1_maketable.txt")
    A = S.pack(np.stack([g["A0"], g["A1"], g["A2"]]))
    T, L = oracle.make_table(A, 8, 0, 3, 0, fix=False)
    Tu = S.unpack(T, 8, 8)
    for idv in range(8):
        key = "T" + format(idv, "03b")
        assert (Tu[L[idv]] == g[key]).all(), key


def test_fig1_add_rows_from_table_golden():
    g = _golden("fig1_maketable.txt")
    A = S.pack(np.stack([g["A0"], g["A1"], g["A2"], g["ROW_BEFORE"]]))
    T, L = oracle.make_table(A, 8, 0, 3, 0, fix=False)
    out = oracle.add_rows_from_table(A, 8, 3, 4, 0, 3, T, L)
    assert (S.unpack(out, 4, 8)[3] == g["ROW_AFTER"]).all()


def test_maketable1_writes_multipliers_golden():
    g = _golden("maketable1_multipliers.txt")
    rng = np.random.default_rng(7)
    for _ in range(20):
        n = 12
        U = np.zeros((4, n), dtype=np.uint8)
        U[0, :3] = g["FIRST_PIVOT_ROW_PREFIX"]
        U[1, 1] = 1
        U[1, 2] = rng.integers(0, 2)
        U[2, 2] = 1
        U[:3, 3:] = rng.integers(0, 2, size=(3, n - 3))
        U[3] = U[0]                          # a row equal to the first pivot row
        U[3, :3] = g["ROW_PREFIX"]
        A = S.pack(U)
        T, L = oracle.make_table(A, n, 0, 3, 0, fix=True)
        out = S.unpack(oracle.add_rows_from_table(A, n, 3, 4, 0, 3, T, L), 4, n)
        assert (out[3, :3] == g["EXPECTED_MULTIPLIERS"]).all()
        assert not out[3, 3:].any()          # cleared by the first pivot row alone


def test_maketable_gray_code_is_all_combinations():
    """T holds every element of the span exactly once, built in 2^k-1 additions."""
    rng = np.random.default_rng(3)
    for k in (1, 2, 4, 6):
        n = 40
        U = np.zeros((k, n), dtype=np.uint8)
        U[:, k:] = rng.integers(0, 2, size=(k, n - k))
        for t in range(k):
            U[t, t] = 1
            U[t, t + 1:k] = rng.integers(0, 2, size=k - t - 1)
        T, L = oracle.make_table(S.pack(U), n, 0, k, 0, fix=False)
        Tu = S.unpack(T, 1 << k, n)
        got = {tuple(r) for r in Tu}
        want = set()
        for mask in range(1 << k):
            v = np.zeros(n, dtype=np.uint8)
            for t in range(k):
                if mask >> t & 1:
                    v ^= U[t]
            want.add(tuple(v))
        assert got == want
        # L maps the id of each row back to it
        for i in range(1 << k):
            idv = int("".join(str(int(b)) for b in Tu[i, :k]), 2)
            assert L[idv] == i


# ----------------------------------------------------------------------------
# rank
# ----------------------------------------------------------------------------

def test_rank_brute_force_span():
    rng = np.random.default_rng(11)
    for _ in range(150):
        m = int(rng.integers(1, 8))
        n = int(rng.integers(1, 9))
        U = (rng.random((m, n)) < rng.choice([0.2, 0.5, 0.8])).astype(np.uint8)
        A = S.pack(U)
        r = oracle.pls(A, m, n)[3]
        assert r == span_rank(U)
        assert oracle.rank(A, m, n) == r


@pytest.mark.parametrize("m,n", [(3, 3), (4, 4), (2, 8), (3, 5), (5, 3)])
def test_rank_exhaustive_closed_form(m, n):
    hist = [0] * (min(m, n) + 1)
    for U in all_matrices(m, n):
        hist[oracle.pls(S.pack(U), m, n)[3]] += 1
    assert hist == [count_rank(m, n, r) for r in range(min(m, n) + 1)]
    if (m, n) == (3, 3):
        assert hist == [1, 49, 294, 168]
    if (m, n) == (4, 4):
        assert hist[4] == 20160


def test_rank_deficiency_distribution_large_square():
    """P(corank d) of a random n x n matrix tends to 0.2888, 0.5776, 0.1284, ..."""
    counts = np.zeros(4)
    N = 600
    for seed in range(N):
        d = 48 - oracle.pls(S.dense(48, 48, seed + 1), 48, 48)[3]
        counts[min(d, 3)] += 1
    freq = counts / N
    expect = np.array([0.2888, 0.5776, 0.1284, 0.0052])
    sigma = np.sqrt(expect * (1 - expect) / N)
    assert (np.abs(freq - expect) < 5 * sigma + 1e-3).all(), freq


# ----------------------------------------------------------------------------
# PLS
# ----------------------------------------------------------------------------

def _inputs(rng, m, n, kind, seed):
    if kind == "dense":
        return S.dense(m, n, seed)
    if kind == "sparse":
        return S.bernoulli(m, n, 0.05, seed)
    if kind == "echelon":
        return S.echelon(m, n, 0.3, seed)
    if kind == "lowrank":
        k = int(rng.integers(1, max(2, min(m, n))))
        return oracle.mul(S.dense(m, k, seed), S.dense(k, n, seed + 7), m, k, n)
    if kind == "zero":
        return S.pack(np.zeros((m, n), dtype=np.uint8))
    raise ValueError(kind)


KINDS = ["dense", "sparse", "echelon", "lowrank", "zero"]


def check_pls_shape(Ain, P, Q, r, m, n):
    A = S.unpack(Ain, m, n) if Ain.dtype == np.uint64 else Ain
    L, Sm = tiny.factors(A, P, Q, r)
    assert 0 <= r <= min(m, n)
    # swap vectors: P[i] >= i, Q strictly increasing on the rank, identity beyond
    assert all(P[i] >= i for i in range(r)) and all(P[i] == i for i in range(r, m))
    assert all(Q[i] < Q[i + 1] for i in range(r - 1)) and all(Q[i] == i for i in range(r, n))
    # L unit lower trapezoidal, S echelon with its leading ones at Q
    for i in range(r):
        assert L[i, i] == 1 and not L[i, i + 1:].any()
        assert Sm[i, Q[i]] == 1 and not Sm[i, :Q[i]].any()
    # stored rows: zeros strictly between the diagonal and the pivot column
    for i in range(r):
        assert not A[i, i + 1:Q[i] + 1 if Q[i] > i else i + 1].any() or Q[i] == i
    # rows past the rank hold only L
    assert not A[r:, r:].any()


@pytest.mark.parametrize("kind", KINDS)
def test_pls_reconstruction_and_shape(kind):
    rng = np.random.default_rng(hash(kind) % 1000)
    for trial in range(40):
        m = int(rng.integers(1, 48))
        n = int(rng.integers(1, 140))
        A = _inputs(rng, m, n, kind, 1000 + trial)
        R, P, Q, r = oracle.pls(A, m, n)
        check_pls_shape(R, P, Q, r, m, n)
        assert (tiny.reconstruct(S.unpack(R, m, n), P, Q, r) == S.unpack(A, m, n)).all()


@pytest.mark.parametrize("kind", KINDS)
def test_pls_matches_independent_restatement(kind):
    rng = np.random.default_rng(5 + len(kind))
    for trial in range(30):
        m = int(rng.integers(1, 65))
        n = int(rng.integers(1, 65))
        A = _inputs(rng, m, n, kind, 2000 + trial)
        R, P, Q, r = oracle.pls(A, m, n)
        T, P2, Q2, r2 = tiny.gauss_pls(S.unpack(A, m, n))
        assert r == r2 and (P == P2).all() and (Q == Q2).all()
        assert (S.unpack(R, m, n) == T).all()


@pytest.mark.parametrize("kind", KINDS)
def test_mmpf_and_recursive_pls_equal_gaussian_pls(kind):
    """The paper's MMPF and recursive PLS give exactly the Gaussian PLS result."""
    rng = np.random.default_rng(17 + len(kind))
    for trial in range(25):
        m = int(rng.integers(1, 70))
        n = int(rng.integers(1, 150))
        A = _inputs(rng, m, n, kind, 3000 + trial)
        ref = oracle.pls(A, m, n)
        k = int(rng.integers(1, 9))
        got = oracle.pls_mmpf(A, m, n, k)
        assert got[3] == ref[3] and (got[1] == ref[1]).all() and (got[2] == ref[2]).all()
        assert (got[0] == ref[0]).all()
        got = oracle.pls_rec(A, m, n, int(rng.integers(1, 40)), k, bool(trial % 2))
        assert got[3] == ref[3] and (got[1] == ref[1]).all() and (got[2] == ref[2]).all()
        assert (got[0] == ref[0]).all()


def test_pls_special_matrices():
    n = 70
    I = S.pack(np.eye(n, dtype=np.uint8))
    R, P, Q, r = oracle.pls(I, n, n)
    assert r == n and (P == np.arange(n)).all() and (Q == np.arange(n)).all() and (R == I).all()
    Z = S.pack(np.zeros((5, 9), dtype=np.uint8))
    R, P, Q, r = oracle.pls(Z, 5, 9)
    assert r == 0 and (R == Z).all() and (P == np.arange(5)).all() and (Q == np.arange(9)).all()
    # a single 1 at (3, 4): pivot found by swapping row 3 up
    U = np.zeros((6, 8), dtype=np.uint8)
    U[3, 4] = 1
    R, P, Q, r = oracle.pls(S.pack(U), 6, 8)
    assert r == 1 and P[0] == 3 and Q[0] == 4
    # all ones m x n: rank 1, every later row keeps L = 1
    O = S.pack(np.ones((7, 13), dtype=np.uint8))
    R, P, Q, r = oracle.pls(O, 7, 13)
    Ru = S.unpack(R, 7, 13)
    assert r == 1 and (Ru[:, 0] == 1).all() and not Ru[1:, 1:].any() and (Ru[0] == 1).all()


# ----------------------------------------------------------------------------
# RREF
# ----------------------------------------------------------------------------

def random_invertible(rng, m):
    while True:
        M = rng.integers(0, 2, size=(m, m)).astype(np.uint8)
        if span_rank(M) == m if m <= 10 else oracle.rank(S.pack(M), m, m) == m:
            return M


def is_rref(R, r):
    m, n = R.shape
    lead = []
    for i in range(r):
        nz = np.nonzero(R[i])[0]
        if nz.size == 0:
            return False
        lead.append(int(nz[0]))
    if any(lead[i] >= lead[i + 1] for i in range(r - 1)):
        return False
    for i, j in enumerate(lead):
        col = R[:, j].copy()
        col[i] = 0
        if col.any():
            return False
    return not R[r:].any()


@pytest.mark.parametrize("kind", KINDS)
def test_rref_unique_idempotent_structured(kind):
    rng = np.random.default_rng(23 + len(kind))
    for trial in range(25):
        m = int(rng.integers(1, 40))
        n = int(rng.integers(1, 100))
        A = _inputs(rng, m, n, kind, 4000 + trial)
        R, piv, r = oracle.rref(A, m, n)
        Ru = S.unpack(R, m, n)
        assert is_rref(Ru, r)
        assert r == oracle.pls(A, m, n)[3]
        # pivots = column rank profile = Q of the PLS decomposition
        assert (piv == oracle.pls(A, m, n)[2][:r]).all()
        # idempotent
        R2, piv2, r2 = oracle.rref(R, m, n)
        assert r2 == r and (R2 == R).all()
        # unique: RREF(M.A) == RREF(A) for invertible M
        M = random_invertible(rng, m)
        MA = oracle.mul(S.pack(M), A, m, m, n)
        R3, _, r3 = oracle.rref(MA, m, n)
        assert r3 == r and (R3 == R).all()
        # every row of A reduces to zero against R (same row space)
        stack = np.vstack([Ru[:r], S.unpack(A, m, n)])
        assert oracle.rank(S.pack(stack), stack.shape[0], n) == r


@pytest.mark.parametrize("kind", KINDS)
def test_m4ri_reaches_the_unique_rref(kind):
    """Algorithm M4RI (Sec. 3.1) gives the reduced row echelon form, which is
    unique (Sec. 2): its result, rank and pivots equal Gauss-Jordan's for every
    table width k, and the structural checks of a reduced echelon form hold."""
    rng = np.random.default_rng(41 + len(kind))
    for trial in range(12):
        m = int(rng.integers(1, 70))
        n = int(rng.integers(1, 140))
        A = _inputs(rng, m, n, kind, 6000 + trial)
        R, piv, r = oracle.rref(A, m, n)
        for k in (1, 2, 3, 5, 8):
            R4, piv4, r4 = oracle.m4ri(A, m, n, k)
            assert r4 == r and (piv4 == piv).all(), (kind, m, n, k)
            W = S.words_per_row(n)
            assert (R4[:, :W] == R[:, :W]).all(), (kind, m, n, k)
            assert is_rref(S.unpack(R4, m, n), r4)


def test_m4ri_worked_example_golden():
    """The M4RI idea of Sec. 3.1 on its printed example (Figure 1): the three
    rows A0..A2 are the identity on the first k = 3 columns, and the row with
    index bits 110 becomes ROW_AFTER once T[110] is added. M4RI with k = 3 on
    [A0; A1; A2; ROW_BEFORE] does exactly that first step; ROW_AFTER is then a
    single 1, so it is the last row of the reduced form, which equals
    Gauss-Jordan's."""
    g = _golden("fig1_maketable.txt")
    M = np.stack([g["A0"], g["A1"], g["A2"], g["ROW_BEFORE"]])
    m, n = M.shape
    assert int(g["ROW_AFTER"].sum()) == 1
    R4, piv4, r4 = oracle.m4ri(S.pack(M), m, n, 3)
    R, piv, r = oracle.rref(S.pack(M), m, n)
    assert r4 == r == 4 and (piv4 == piv).all() and (R4 == R).all()
    assert (S.unpack(R4, m, n)[3] == g["ROW_AFTER"]).all()


def test_rref_special_matrices():
    n = 20
    I = np.eye(n, dtype=np.uint8)
    R, piv, r = oracle.rref(S.pack(I), n, n)
    assert r == n and (S.unpack(R, n, n) == I).all()
    perm = np.random.default_rng(1).permutation(n)
    R, piv, r = oracle.rref(S.pack(I[perm]), n, n)
    assert r == n and (S.unpack(R, n, n) == I).all()
    R, piv, r = oracle.rref(S.pack(np.zeros((4, 7), np.uint8)), 4, 7)
    assert r == 0 and not R.any()


# ----------------------------------------------------------------------------
# product
# ----------------------------------------------------------------------------

def test_mul_matches_integer_matmul_mod2():
    rng = np.random.default_rng(9)
    for _ in range(30):
        m, k, n = (int(x) for x in rng.integers(1, 150, size=3))
        A = rng.integers(0, 2, size=(m, k)).astype(np.uint8)
        B = rng.integers(0, 2, size=(k, n)).astype(np.uint8)
        C0 = rng.integers(0, 2, size=(m, n)).astype(np.uint8)
        want = (A.astype(np.int64) @ B.astype(np.int64)) % 2
        got = S.unpack(oracle.mul(S.pack(A), S.pack(B), m, k, n), m, n)
        assert (got == want).all()
        got = S.unpack(oracle.mul(S.pack(A), S.pack(B), m, k, n, C=S.pack(C0)), m, n)
        assert (got == (want ^ C0)).all()


# ----------------------------------------------------------------------------
# planted mistakes: each plausible slip in the C oracle fails a pin above
# ----------------------------------------------------------------------------

MUTANTS = {
    # eliminate from column j instead of j+1: L is lost
    "l_lost": ("add_row_from(A, s, n, l, r, pj + 1);", "add_row_from(A, s, n, l, r, pj);"),
    # no compression of L
    "no_compress": ("swap_cols_from(A, s, m, j, Q[j], j);", "(void)0;"),
    # compress from row 0 instead of row j
    "compress_row0": ("swap_cols_from(A, s, m, j, Q[j], j);", "swap_cols_from(A, s, m, j, Q[j], 0);"),
    # search by rows first (pivot rule changed)
    "row_first": ("for (int64_t j = c; j < n && pi < 0; ++j) {\n            for (int64_t i = r; i < m; ++i) {\n                if (getb(A, s, i, j)) {",
                  "for (int64_t i = r; i < m && pi < 0; ++i) {\n            for (int64_t j = c; j < n; ++j) {\n                if (getb(A, s, i, j)) {"),
    # Gauss-Jordan forgetting the rows above (REF instead of RREF)
    "ref_only": ("if (l != r && getb(A, s, l, j))", "if (l > r && getb(A, s, l, j))"),
    # product ignoring the accumulate flag
    "mul_noacc": ("if (!acc)\n            memset", "if (1)\n            memset"),
    # MakeTable1 without the a-priori id fix
    "no_fix": ("    if (fix) {\n        for (int64_t i = 1; i < N; ++i) {", "    if (0) {\n        for (int64_t i = 1; i < N; ++i) {"),
    # M4RI clearing only the rows below the block (an echelon form, not the reduced one)
    "m4ri_below_only": ("vadd_rows_from_table(V, 0, r, c, kbar, T, L);", "(void)0;"),
    # GaussSubmatrix without clearing above its pivots (the block is not the identity)
    "gauss_submatrix_no_above": ("for (int64_t l = r; l < rs; ++l)\n                    if (vget(A, l, j))",
                                 "for (int64_t l = rs; l < rs; ++l)\n                    if (vget(A, l, j))"),
}


def _build_mutant(tmp_path, name):
    import ctypes
    import subprocess
    src = open(os.path.join(os.path.dirname(oracle.__file__), "gf2_oracle.c")).read()
    old, new = MUTANTS[name]
    assert old in src, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path)])
    return ctypes.CDLL(str(so))


def _pins_pass(lib) -> bool:
    """Run a quick subset of the pins against a (possibly mutated) library."""
    import ctypes
    saved = oracle._lib
    lib.gf2o_pls.restype = ctypes.c_int64
    lib.gf2o_rref.restype = ctypes.c_int64
    lib.gf2o_pls_mmpf.restype = ctypes.c_int64
    lib.gf2o_pls_rec.restype = ctypes.c_int64
    lib.gf2o_m4ri.restype = ctypes.c_int64
    for f in ("gf2o_pls", "gf2o_rref", "gf2o_mul", "gf2o_pls_mmpf", "gf2o_pls_rec", "gf2o_m4ri",
              "gf2o_make_table", "gf2o_add_rows_from_table"):
        getattr(lib, f).argtypes = getattr(oracle._load(), f).argtypes
    oracle._lib = lib
    try:
        test_maketable1_writes_multipliers_golden()
        test_mul_matches_integer_matmul_mod2()
        for kind in KINDS:
            test_pls_reconstruction_and_shape(kind)
            test_pls_matches_independent_restatement(kind)
        test_rref_unique_idempotent_structured("dense")
        test_m4ri_reaches_the_unique_rref("dense")
        test_rank_brute_force_span()
        return True
    except AssertionError:
        return False
    finally:
        oracle._lib = saved


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert _pins_pass(oracle._load())
    assert not _pins_pass(_build_mutant(tmp_path, name)), f"mutant {name} passed the pins"
