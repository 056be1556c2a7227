#!/usr/bin/env python3
"""Write SHA-256 digests of the oracle's results at the benchmark's full sizes.

Calls only ``oracle/`` (Gaussian PLS of the appendix, Gauss-Jordan RREF, the
product by definition) on inputs from the host generator ``synth.py``, which
the device generator reproduces bit for bit. Output:
``tests/golden/fullsize_digests.json``, read by ``tests/test_gpu_digests.py``.

Cases:
* ``c3_dense``, ``c3_product``, ``c3_sparse01`` -- the three 65536 x 65536
  matrices: Bernoulli(1/2); A = B.C with B 65536 x 32768 and C 32768 x 65536
  dense (A formed by ``oracle.mul``); Bernoulli(0.01);
* ``c4_<i>`` -- every member i with m >= 4096 of the 2048-matrix batch;
* ``c5_<i>`` -- 16 requests of the 4096-request stream (a seeded draw plus the
  largest), echelon-structured.

For each case: m, n, rank, and the digests of the input, of P and Q (int64,
lengths m and n), of the in-place PLS result (words [0, ceil(n/64)) of every
row), of the RREF (same words) and of its pivot columns (int64, length r).

  python tests/golden/make_fullsize_digests.py [--jobs 8] [--only c3,c4,c5]

Single-threaded oracle per case; cases run in parallel processes (spawned).
The 65536 x 65536 cases take about half an hour each on one core.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "fullsize_digests.json")
SEED = 0x10061744


def digest(a) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def make_input(case: dict):
    """The case's input matrix from the host generator (and the oracle's product for A = B.C)."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    from paper_1006_1744_gb300 import synth as S
    kind, m, n = case["kind"], case["m"], case["n"]
    if kind == "dense":
        return S.dense(m, n, case["seed"])
    if kind == "bernoulli":
        return S.bernoulli(m, n, case["p"], case["seed"])
    if kind == "product":
        k = case["k"]
        B = S.dense(m, k, case["seed_b"])
        C = S.dense(k, n, case["seed_c"])
        return oracle.mul(B, C, m, k, n)
    if kind == "echelon":
        return S.echelon(m, n, case["p"], case["seed"], frac=case["frac"])
    raise ValueError(kind)


def run_case(case: dict) -> dict:
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    m, n = case["m"], case["n"]
    W = (n + 63) // 64
    t0 = time.time()
    A = make_input(case)
    out = dict(case)
    out["input"] = digest(A[:, :W])
    R, P, Q, r = oracle.pls(A, m, n)
    out.update({"rank": r, "P": digest(P.astype(np.int64)), "Q": digest(Q.astype(np.int64)),
                "pls": digest(R[:, :W])})
    del R
    RR, piv, rr = oracle.rref(A, m, n)
    assert rr == r
    out.update({"rref": digest(RR[:, :W]), "pivots": digest(piv.astype(np.int64))})
    out["oracle_seconds"] = time.time() - t0
    return out


def cases(only: set[str]) -> list[dict]:
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import numpy as np
    from paper_1006_1744_gb300 import synth as S
    out = []
    if "c3" in only:
        n = 65536
        out.append({"name": "c3_product", "kind": "product", "m": n, "n": n, "k": 32768,
                    "seed_b": SEED + 3, "seed_c": SEED + 4})
        out.append({"name": "c3_dense", "kind": "dense", "m": n, "n": n, "seed": SEED})
        out.append({"name": "c3_sparse01", "kind": "bernoulli", "m": n, "n": n, "p": 0.01, "seed": SEED + 2})
    if "c5" in only:
        rec = S.request_recipe(4096, SEED)
        big = max(range(len(rec)), key=lambda i: rec[i][0] * rec[i][1])
        rng = np.random.default_rng(5)
        pick = sorted(set(rng.choice(len(rec), 15, replace=False).tolist()) | {big})
        for i in pick:
            m, n, sd = rec[i]
            out.append({"name": f"c5_{i}", "kind": "echelon", "m": m, "n": n, "p": 0.3, "frac": 0.5, "seed": sd,
                        "index": i})
    if "c4" in only:
        rec = S.batch_recipe(2048, SEED)
        for i, (m, n, p, sd) in enumerate(rec):
            if m >= 4096:
                kind = "dense" if p == 0.5 else "bernoulli"
                out.append({"name": f"c4_{i}", "kind": kind, "m": m, "n": n, "p": p, "seed": sd, "index": i})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", default="c3,c4,c5")
    args = ap.parse_args()
    todo = cases(set(args.only.split(",")))
    have = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            have = {c["name"]: c for c in json.load(f)["cases"]}
    todo = [c for c in todo if c["name"] not in have]
    # largest first, so that the long cases start at once
    todo.sort(key=lambda c: -c["m"] * c["n"] * (3 if c["kind"] == "product" else 1))
    print(f"{len(todo)} cases to run, {len(have)} done", flush=True)
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        for res in pool.imap_unordered(run_case, todo):
            have[res["name"]] = res
            with open(OUT + ".tmp", "w") as f:
                json.dump({"seed": SEED, "generator": "paper_1006_1744_gb300/synth.py",
                           "oracle": "oracle/gf2_oracle.c (gf2o_pls, gf2o_rref, gf2o_mul)",
                           "cases": sorted(have.values(), key=lambda c: c["name"])}, f, indent=0)
            os.replace(OUT + ".tmp", OUT)
            print(f"{res['name']}: rank {res['rank']} ({res['oracle_seconds']:.1f} s)", flush=True)


if __name__ == "__main__":
    main()
