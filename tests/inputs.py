"""Seeded test inputs of the shapes the paper's workloads have (dense random,
sparse, staircase, low rank, degenerate). Only data generation: no elimination
arithmetic except ``lowrank``, whose product is taken by the oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1006_1744_gb300 import synth as S

KINDS = ["dense", "sparse05", "sparse01", "echelon", "lowrank", "deep", "dup", "zero", "identity", "ones"]


def make(kind: str, m: int, n: int, seed: int, stride: int | None = None) -> np.ndarray:
    stride = S.default_stride(n) if stride is None else stride
    if kind == "dense":
        return S.dense(m, n, seed, stride)
    if kind == "sparse05":
        return S.bernoulli(m, n, 0.05, seed, stride)
    if kind == "sparse01":
        return S.bernoulli(m, n, 0.01, seed, stride)
    if kind == "echelon":
        return S.echelon(m, n, 0.3, seed, stride=stride)
    if kind == "lowrank":
        k = max(1, min(m, n) // 2)
        B = S.dense(m, k, S.derive_seed(seed, 1))
        C = S.dense(k, n, S.derive_seed(seed, 2))
        return oracle.mul(B, C, m, k, n, stride=stride)
    if kind == "deep":
        # the first 300 rows are zero: every pivot search must look past the window
        A = S.dense(m, n, seed, stride)
        A[:min(m, 300)] = 0
        return A
    if kind == "dup":
        # only 5 distinct rows
        base = S.dense(5, n, seed, stride)
        idx = np.random.default_rng(seed).integers(0, 5, size=m)
        return base[idx].copy()
    if kind == "zero":
        return np.zeros((m, stride), dtype=np.uint64)
    if kind == "identity":
        U = np.zeros((m, n), dtype=np.uint8)
        d = min(m, n)
        U[np.arange(d), np.arange(d)] = 1
        return S.pack(U, stride)
    if kind == "ones":
        return S.pack(np.ones((m, n), dtype=np.uint8), stride)
    raise ValueError(kind)
