"""Full-size parity: the GPU path against the oracle's SHA-256 digests.

``tests/golden/fullsize_digests.json`` holds, for every full-size workload the
benchmark times, the digests of the oracle's results (Gaussian PLS of the
appendix, Gauss-Jordan RREF; written by ``tests/golden/make_fullsize_digests.py``,
which calls only ``oracle/``): rank, P, Q, the in-place PLS matrix, the RREF and
its pivot columns, plus the digest of the input itself. Here the same inputs are
made by the device generator and every GPU route is compared with them:

* the three 65536 x 65536 matrices (dense; A = B.C formed on the GPU by both
  product forms; Bernoulli(0.01)) through gf2_pls by MMPF panels and by the
  recursive PLS with the XOR-table and the tensor-core product (cutoff 4096
  columns), and through gf2_rref by the PLS route, by M4RI and by the hybrid;
* every member with m >= 4096 of the 2048-matrix batch, through one
  gf2_pls_batched call and through gf2_rref;
* 16 requests of the request stream (the largest included), through gf2_pls,
  one gf2_pls_batched call over all 16, and gf2_rref.
MMPF and the recursive PLS reach the Gaussian PLS result exactly (Sec. 4, 5),
and the RREF is unique, so every digest must match.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

from paper_1006_1744_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
DIGESTS = os.path.join(HERE, "golden", "fullsize_digests.json")


def _cases():
    if not os.path.exists(DIGESTS):
        return {}
    with open(DIGESTS) as f:
        return {c["name"]: c for c in json.load(f)["cases"]}


CASES = _cases()


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_1744_gb300 import build, gf2
    build.build()
    return gf2


def sha(a) -> str:
    if isinstance(a, torch.Tensor):
        a = a.cpu().numpy()
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def words(t, n) -> np.ndarray:
    """Host copy of the words [0, ceil(n/64)) of every row (uint64)."""
    return t.cpu().numpy().view(np.uint64)[:, :S.words_per_row(n)]


def make_input(case, dev="cuda"):
    from paper_1006_1744_gb300 import synth_gpu
    m, n = case["m"], case["n"]
    A = torch.empty((m, S.default_stride(n)), dtype=torch.int64, device=dev)
    kind = case["kind"]
    if kind == "dense":
        synth_gpu.fill(A, n, case["seed"])
    elif kind == "bernoulli":
        synth_gpu.fill(A, n, case["seed"], p=case["p"])
    elif kind == "echelon":
        synth_gpu.fill(A, n, case["seed"], p=case["p"], echelon_frac=case["frac"])
    else:
        raise ValueError(kind)
    return A


def check_pls(case, A, P, Q, rank, n, what):
    m = case["m"]
    assert int(rank) == case["rank"], (what, int(rank), case["rank"])
    assert sha(P[:m]) == case["P"], (what, "P")
    assert sha(Q[:n]) == case["Q"], (what, "Q")
    assert sha(words(A, n)) == case["pls"], (what, "in-place PLS matrix")


def check_rref(case, A, rank, piv, n, what):
    r = case["rank"]
    assert int(rank) == r, (what, int(rank), r)
    assert sha(piv[:r]) == case["pivots"], (what, "pivots")
    assert sha(words(A, n)) == case["rref"], (what, "RREF")


C3 = [k for k in ("c3_dense", "c3_product", "c3_sparse01") if k in CASES]


@pytest.mark.parametrize("name", C3)
def test_65536_against_oracle_digests(g, name):
    case = CASES[name]
    n = case["n"]
    if case["kind"] == "product":
        from paper_1006_1744_gb300 import synth_gpu
        k = case["k"]
        B = torch.empty((n, S.default_stride(k)), dtype=torch.int64, device="cuda")
        C = torch.empty((k, S.default_stride(n)), dtype=torch.int64, device="cuda")
        synth_gpu.fill(B, k, case["seed_b"])
        synth_gpu.fill(C, n, case["seed_c"])
        A0 = torch.empty((n, S.default_stride(n)), dtype=torch.int64, device="cuda")
        for product in (g.PRODUCT_XOR, g.PRODUCT_TENSOR):
            g.mul(A0, B, C, n, k, n, opts={"product": product})
            torch.cuda.synchronize()
            assert sha(words(A0, n)) == case["input"], ("A = B.C", product)
        del B, C
        torch.cuda.empty_cache()
    else:
        A0 = make_input(case)
        assert sha(words(A0, n)) == case["input"], "device generator"
    A = torch.empty_like(A0)
    for what, opts in (("MMPF", None), ("recursive, XOR product", {"cutoff_cols": 4096, "product": 1}),
                       ("recursive, tensor-core product", {"cutoff_cols": 4096, "product": 2})):
        A.copy_(A0)
        P, Q, rk = g.pls(A, n, opts=opts)
        torch.cuda.synchronize()
        check_pls(case, A, P, Q, rk.item(), n, what)
        del P, Q
    for what, meth in (("RREF, PLS route", g.RREF_PLS), ("RREF, M4RI", g.RREF_M4RI),
                       ("RREF, hybrid", g.RREF_HYBRID)):
        A.copy_(A0)
        rk, piv = g.rref(A, n, opts={"rref_method": meth})
        torch.cuda.synchronize()
        check_rref(case, A, rk.item(), piv, n, what)
    del A, A0
    torch.cuda.empty_cache()


C4 = sorted((c for c in CASES.values() if c["name"].startswith("c4_")), key=lambda c: c["index"])


@pytest.mark.skipif(not C4, reason="no batch digests")
def test_batch_members_against_oracle_digests(g):
    """The whole 2048-matrix batch in one gf2_pls_batched call (default options); every
    member with m >= 4096 against its digests, then through gf2_rref (all three routes)."""
    from paper_1006_1744_gb300 import synth_gpu
    rec = S.batch_recipe(2048, 0x10061744)
    mats, ns = [], []
    for (m, n, p, sd) in rec:
        D = torch.empty((m, S.default_stride(n)), dtype=torch.int64, device="cuda")
        synth_gpu.fill(D, n, sd, p=p)
        mats.append(D)
        ns.append(n)
    orig = {c["index"]: mats[c["index"]].clone() for c in C4}
    for c in C4:
        assert sha(words(orig[c["index"]], c["n"])) == c["input"], c["name"]
    Ps, Qs, ranks = g.pls_batched(mats, ns)
    torch.cuda.synchronize()
    rk = ranks.cpu().numpy()
    for c in C4:
        i = c["index"]
        check_pls(c, mats[i], Ps[i], Qs[i], rk[i], c["n"], c["name"])
    for c in C4:
        i = c["index"]
        for meth in (g.RREF_PLS, g.RREF_M4RI, g.RREF_HYBRID):
            A = orig[i].clone()
            r, piv = g.rref(A, c["n"], opts={"rref_method": meth})
            torch.cuda.synchronize()
            check_rref(c, A, r.item(), piv, c["n"], (c["name"], meth))


C5 = sorted((c for c in CASES.values() if c["name"].startswith("c5_")), key=lambda c: c["index"])


@pytest.mark.skipif(not C5, reason="no request digests")
def test_request_stream_sample_against_oracle_digests(g):
    """16 echelon-structured requests (the largest included): each through gf2_pls, all 16 in
    one gf2_pls_batched call, and each through gf2_rref's three routes."""
    origs = [make_input(c) for c in C5]
    for c, A0 in zip(C5, origs):
        assert sha(words(A0, c["n"])) == c["input"], c["name"]
    for c, A0 in zip(C5, origs):
        A = A0.clone()
        P, Q, rk = g.pls(A, c["n"])
        torch.cuda.synchronize()
        check_pls(c, A, P, Q, rk.item(), c["n"], (c["name"], "gf2_pls"))
        for meth in (g.RREF_PLS, g.RREF_M4RI, g.RREF_HYBRID):
            A = A0.clone()
            r, piv = g.rref(A, c["n"], opts={"rref_method": meth})
            torch.cuda.synchronize()
            check_rref(c, A, r.item(), piv, c["n"], (c["name"], meth))
    mats = [A0.clone() for A0 in origs]
    Ps, Qs, ranks = g.pls_batched(mats, [c["n"] for c in C5])
    torch.cuda.synchronize()
    rk = ranks.cpu().numpy()
    for i, c in enumerate(C5):
        check_pls(c, mats[i], Ps[i], Qs[i], rk[i], c["n"], (c["name"], "batched"))
