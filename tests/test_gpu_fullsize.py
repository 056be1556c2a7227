"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (default options, the benchmark's seed):

* 16384 x 16384 dense: gf2_pls and gf2_rref bit for bit against the oracle;
* 65536 x 65536 dense: the decomposition checked by its definition,
  A.x = P.L.S.x for random vectors x (Freivalds), L and S read from the
  in-place result;
* the 2048-matrix batch: a seeded sample of its matrices against the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1006_1744_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED = 0x10061744
POP8 = np.array([bin(i).count("1") & 1 for i in range(256)], dtype=np.uint8)


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_1744_gb300 import build, gf2
    build.build()
    return gf2


def host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def test_headline_16384_pls_and_rref_bit_exact(g):
    from paper_1006_1744_gb300 import synth_gpu
    n = 16384
    A0 = synth_gpu.dense(n, n, SEED)
    Ah = host(A0)
    assert (Ah == S.dense(n, n, SEED)).all()  # the device generator is the host recipe
    R, P, Q, r = oracle.pls(Ah, n, n)
    A = A0.clone()
    Pd, Qd, rd = g.pls(A, n)
    torch.cuda.synchronize()
    assert int(rd.item()) == r
    assert (Pd.cpu().numpy() == P).all() and (Qd.cpu().numpy() == Q).all()
    W = S.words_per_row(n)
    assert (host(A)[:, :W] == R[:, :W]).all()
    Rr, piv, rr = oracle.rref(Ah, n, n)
    A2 = A0.clone()
    rank2, pivd = g.rref(A2, n)
    torch.cuda.synchronize()
    assert int(rank2.item()) == rr
    assert (pivd.cpu().numpy()[:rr] == piv).all()
    assert (host(A2)[:, :W] == Rr[:, :W]).all()


def _parity_rows(M, x):
    """(M & x) parity per row, M (rows, W) uint64, x (W,) uint64 -> uint8."""
    t = (M & x[None, :]).view(np.uint8).reshape(M.shape[0], -1)
    return np.bitwise_xor.reduce(POP8[t], axis=1).astype(np.uint8)


def _mask_gt(th, W):
    """Per row, the bits of the columns > th[row]."""
    widx = np.arange(W)[None, :]
    wq = (th >> 6)[:, None]
    full = np.where(widx > wq, np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0))
    part = ~((np.uint64(2) << (th & 63).astype(np.uint64)[:, None]) - np.uint64(1))
    return np.where(widx == wq, part, full)


def _mask_lt(lim, W):
    """Per row, the bits of the columns < lim[row]."""
    widx = np.arange(W)[None, :]
    wq = (lim >> 6)[:, None]
    full = np.where(widx < wq, np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0))
    part = (np.uint64(1) << (lim & 63).astype(np.uint64)[:, None]) - np.uint64(1)
    return np.where(widx == wq, part, full)


def _pack(bits, W):
    out = np.zeros(W * 64, dtype=np.uint8)
    out[:bits.size] = bits
    return np.packbits(out, bitorder="little").view(np.uint64)


def test_65536_decomposition_by_definition(g):
    """A.x == P.(L.(S.x)) for random x, with L (unit lower trapezoidal) and S
    (echelon, leading ones at Q) read from the in-place result as the header
    specifies; also the structural facts (Q increasing, L's diagonal implied)."""
    from paper_1006_1744_gb300 import synth_gpu
    n = m = 65536
    W = S.words_per_row(n)
    A0 = synth_gpu.dense(m, n, SEED)
    A = A0.clone()
    Pd, Qd, rd = g.pls(A, n)
    torch.cuda.synchronize()
    r = int(rd.item())
    P = Pd.cpu().numpy()
    Q = Qd.cpu().numpy()
    assert r > m - 20
    assert (np.diff(Q[:r]) > 0).all()  # pivot columns increase
    Ah, Rh = host(A0)[:, :W], host(A)[:, :W]
    del A, A0
    torch.cuda.empty_cache()
    rng = np.random.default_rng(3)
    for _ in range(2):
        xb = rng.integers(0, 2, n, dtype=np.uint8)
        x = _pack(xb, W)
        ax = _parity_rows(Ah, x)
        # S.x: row i < r is a 1 at Q[i] plus the stored bits right of Q[i]
        sx = np.zeros(r, dtype=np.uint8)
        for i0 in range(0, r, 4096):
            i1 = min(r, i0 + 4096)
            q = Q[i0:i1]
            sx[i0:i1] = _parity_rows(Rh[i0:i1] & _mask_gt(q, W), x) ^ xb[q]
        # L.(S.x): row i holds the multipliers in columns < min(i, r), unit diagonal for i < r
        y = _pack(sx, W)
        lsx = np.zeros(m, dtype=np.uint8)
        for i0 in range(0, m, 4096):
            i1 = min(m, i0 + 4096)
            lim = np.minimum(np.arange(i0, i1, dtype=np.int64), r)
            lsx[i0:i1] = _parity_rows(Rh[i0:i1] & _mask_lt(lim, W), y)
        lsx[:r] ^= sx
        # P: the swaps i <-> P[i] for i = r-1 down to 0
        v = lsx.copy()
        for i in range(r - 1, -1, -1):
            pi = P[i]
            if pi != i:
                v[i], v[pi] = v[pi], v[i]
        assert np.array_equal(v, ax)


def test_batch_sample_against_oracle(g):
    """The 2048-matrix batch through one gf2_pls_batched call (default options);
    24 of its matrices, chosen by a seeded draw, compared with the oracle."""
    from paper_1006_1744_gb300 import synth_gpu
    rec = S.batch_recipe(2048, SEED)
    mats, ns = [], []
    for (m, n, p, sd) in rec:
        D = torch.empty((m, S.default_stride(n)), dtype=torch.int64, device="cuda")
        synth_gpu.fill(D, n, sd, p=p)
        mats.append(D)
        ns.append(n)
    rng = np.random.default_rng(11)
    small = [i for i, (m, n, p, sd) in enumerate(rec) if m * n <= 2048 * 4096]
    pick = sorted(rng.choice(small, 24, replace=False).tolist())
    orig = {i: host(mats[i]).copy() for i in pick}
    Ps, Qs, ranks = g.pls_batched(mats, ns)
    torch.cuda.synchronize()
    rk = ranks.cpu().numpy()
    for i in pick:
        m, n, p, sd = rec[i]
        R, P, Q, r = oracle.pls(orig[i], m, n)
        assert rk[i] == r, i
        assert (Ps[i].cpu().numpy()[:m] == P[:m]).all(), i
        assert (Qs[i].cpu().numpy()[:n] == Q[:n]).all(), i
        W = S.words_per_row(n)
        assert (host(mats[i])[:, :W] == R[:, :W]).all(), i
