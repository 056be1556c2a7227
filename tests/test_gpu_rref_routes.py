"""The direct reduced-echelon routes of gf2_rref against the oracle.

* Algorithm M4RI (Sec. 3.1; GF2_RREF_M4RI): each panel's tables clear the
  rows above and below; the result must be the oracle's (Gauss-Jordan) RREF,
  which is unique (Definition "Reduced Row Echelon Form"), bit for bit, with
  the same rank and pivot columns.
* The hybrid "M+P" (Sec. 6-7; GF2_RREF_HYBRID): reduced-form panels while the
  remaining rows' density stays below the threshold, PLS panels and the upper
  solve after; thresholds that switch at once, at the paper's 0.15, and never.
Inputs: every kind of tests/inputs.py over shapes with ragged tails, tall and
wide, rank-deficient, and row pitches wider than the minimum.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1006_1744_gb300 import synth as S
from tests.inputs import KINDS, make

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(1, 1), (1, 64), (64, 1), (7, 13), (64, 64), (65, 65), (100, 200), (200, 100), (128, 129),
          (129, 300), (257, 257), (300, 64), (500, 700), (700, 500), (1024, 1024), (1300, 2100)]


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_1744_gb300 import build, gf2
    build.build()
    return gf2


def _check(g, A, m, n, opts, stride=None):
    R, piv, r = oracle.rref(A, m, n)
    W = S.words_per_row(n)
    stride = A.shape[1] if stride is None else stride
    Aw = np.zeros((m, stride), dtype=np.uint64)
    Aw[:, :W] = A[:, :W]
    if stride > W:
        Aw[:, W:] = np.uint64(0x5A5A5A5A5A5A5A5A)  # words past the row must stay untouched
    D = torch.from_numpy(Aw.view(np.int64)).cuda()
    rd, pd = g.rref(D, n, opts=opts)
    torch.cuda.synchronize()
    assert int(rd.item()) == r
    assert (pd.cpu().numpy()[:r] == piv).all(), "pivot columns differ"
    assert (pd.cpu().numpy()[r:n] == np.arange(r, n)).all()
    got = D.cpu().numpy().view(np.uint64)
    bad = np.nonzero((got[:, :W] != R[:, :W]).any(axis=1))[0]
    assert bad.size == 0, f"rows differ: {bad[:10]}"
    if stride > W:
        assert (got[:, W:] == np.uint64(0x5A5A5A5A5A5A5A5A)).all()


@pytest.mark.parametrize("kind", KINDS)
def test_rref_m4ri_parity(g, kind):
    for i, (m, n) in enumerate(SHAPES):
        _check(g, make(kind, m, n, 900 + i), m, n, {"rref_method": g.RREF_M4RI})


@pytest.mark.parametrize("permille", [1, 150, 1000])
@pytest.mark.parametrize("kind", KINDS)
def test_rref_hybrid_parity(g, kind, permille):
    for i, (m, n) in enumerate(SHAPES):
        _check(g, make(kind, m, n, 1900 + i), m, n, {"rref_method": g.RREF_HYBRID, "hybrid_permille": permille})


@pytest.mark.parametrize("method", ["M4RI", "HYBRID"])
def test_rref_routes_wide_stride_and_rank_deficient(g, method):
    opts = {"rref_method": getattr(g, "RREF_" + method)}
    for (m, n, stride) in [(700, 900, 32), (300, 500, 48), (129, 64, 32), (2100, 700, 16), (300, 2000, 48)]:
        for kind in ("dense", "lowrank", "echelon", "sparse01", "deep"):
            _check(g, make(kind, m, n, 3 * m + stride), m, n, opts, stride=stride)


def test_rref_hybrid_switches_on_sparse_then_dense_input(g):
    """An input that starts sparse (1%) and fills in: the hybrid runs reduced-form panels
    first and PLS panels later, with the upper solve over the later pivots only."""
    m, n = 2000, 3000
    A = make("sparse01", m, n, 77)
    for permille in (100, 150, 200, 400):
        _check(g, A, m, n, {"rref_method": g.RREF_HYBRID, "hybrid_permille": permille})


def test_rref_routes_reject_other_tiles(g):
    A = torch.zeros((64, 16), dtype=torch.int64, device="cuda")
    with pytest.raises(g.Gf2Error):
        g.rref(A, 64, opts={"rref_method": g.RREF_M4RI, "tile_words": 8})
