"""Two panels per table sweep (``panels_per_sweep = 2``): the pivots of panels b
and b + 1 first, then one sweep of the trailing block for both (MMPF, Sec. 4.1,
with 128 pivot columns per AddRowsFromTable pass). The elimination is the same
Gaussian PLS, so rank, P, Q, the in-place PLS matrix, the RREF (PLS route) and
the rank must equal the oracle's bit for bit on every input kind: odd and even
panel counts, ragged last words, pivot searches past the window (row-order
changes deferred by one panel), rank deficiency (panels without pivots, the
zero-tail test four panels later), and grids of any size."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1006_1744_gb300 import synth as S

from tests.inputs import KINDS, make

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PAIR = {"panels_per_sweep": 2}

# panel counts 1..33 (odd and even), tiles and 128-byte lines split at every offset
SHAPES = [(1, 1), (7, 13), (64, 64), (65, 129), (129, 65), (128, 192), (200, 130), (300, 256), (257, 300),
          (500, 700), (700, 500), (1024, 1024), (1100, 1150), (640, 2100), (2100, 640)]


def dev(A: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(A).view(np.int64)).cuda()


def host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_1744_gb300 import build, gf2
    build.build()
    return gf2


def check_pls(g, A, m, n, opts):
    R, P, Q, r = oracle.pls(A, m, n)
    D = dev(A)
    Pd, Qd, rd = g.pls(D, n, opts=opts)
    torch.cuda.synchronize()
    assert int(rd.item()) == r, (m, n, int(rd.item()), r)
    assert (Pd.cpu().numpy() == P).all(), "P differs"
    assert (Qd.cpu().numpy() == Q).all(), "Q differs"
    W = S.words_per_row(n)
    bad = np.nonzero((host(D)[:, :W] != R[:, :W]).any(axis=1))[0]
    assert bad.size == 0, f"rows differ: {bad[:10]}"
    return r


@pytest.mark.parametrize("kind", KINDS)
def test_pair_pls_parity_shapes(g, kind):
    for i, (m, n) in enumerate(SHAPES):
        A = make(kind, m, n, 5100 + i)
        check_pls(g, A, m, n, PAIR)


@pytest.mark.parametrize("kind", ["dense", "deep", "lowrank", "echelon", "sparse01"])
def test_pair_rank_and_rref_parity(g, kind):
    for i, (m, n) in enumerate([(65, 129), (300, 256), (700, 500), (1100, 1150), (640, 2100)]):
        A = make(kind, m, n, 5300 + i)
        assert int(g.rank(dev(A), n, opts=PAIR).item()) == oracle.rank(A, m, n)
        R, piv, r = oracle.rref(A, m, n)
        D = dev(A)
        rd, pd = g.rref(D, n, opts=dict(PAIR, rref_method=g.RREF_PLS))
        torch.cuda.synchronize()
        assert int(rd.item()) == r
        assert (pd.cpu().numpy()[:r] == piv).all()
        W = S.words_per_row(n)
        assert (host(D)[:, :W] == R[:, :W]).all()


@pytest.mark.parametrize("grid", [1, 2, 3, 17, 152, 400])
def test_pair_grid_choices(g, grid):
    for kind in ("dense", "deep", "lowrank"):
        A = make(kind, 900, 1300, grid)
        check_pls(g, A, 900, 1300, dict(PAIR, grid_ctas=grid))


def test_pair_zero_tail_and_wide_rank_deficiency(g):
    """Rank 96 in 40 panels: after the pivots run out, panels with no pivot test the rest
    of the trailing block for a nonzero word and later searches skip their windows."""
    m, n, k = 700, 2560, 96
    B = S.dense(m, k, 11)
    C = S.dense(k, n, 12)
    A = oracle.mul(B, C, m, k, n)
    assert check_pls(g, A, m, n, PAIR) == k
    # nonzero columns only far to the right of a zero block
    A2 = np.zeros((m, S.default_stride(n)), dtype=np.uint64)
    A2[:, 30] = S.dense(m, 64, 13)[:, 0]
    check_pls(g, A2, m, n, PAIR)


def test_pair_same_as_one_panel_at_size(g):
    """Several thousand rows: both pipelines against the oracle on the same inputs."""
    for kind, seed in (("dense", 1), ("sparse05", 2), ("lowrank", 3)):
        A = make(kind, 3000, 3100, 5400 + seed)
        r2 = check_pls(g, A, 3000, 3100, PAIR)
        r1 = check_pls(g, A, 3000, 3100, {"panels_per_sweep": 1})
        assert r1 == r2


def test_pair_replayed_calls_with_new_contents(g):
    """Repeated calls on the same buffers run as graph replays; the contents change."""
    m, n = 800, 1000
    D = torch.empty((m, S.default_stride(n)), dtype=torch.int64, device="cuda")
    P = torch.empty(m, dtype=torch.int64, device="cuda")
    Q = torch.empty(n, dtype=torch.int64, device="cuda")
    rank = torch.empty(1, dtype=torch.int64, device="cuda")
    for i in range(5):
        A = make(["dense", "deep", "lowrank", "dense", "echelon"][i], m, n, 5500 + i)
        R, Pw, Qw, r = oracle.pls(A, m, n)
        D.copy_(dev(A))
        g.pls(D, n, P=P, Q=Q, rank=rank, opts=PAIR)
        torch.cuda.synchronize()
        assert int(rank.item()) == r
        assert (P.cpu().numpy() == Pw).all() and (Q.cpu().numpy() == Qw).all()
        W = S.words_per_row(n)
        assert (host(D)[:, :W] == R[:, :W]).all()


def test_pair_more_rows_than_front_threads(g):
    """More rows than the front kernel has threads (152 CTAs x 512): each thread takes a
    second row after the tables are built."""
    for kind, (m, n) in (("dense", (100000, 300)), ("lowrank", (90000, 200)), ("echelon", (81000, 450))):
        A = make(kind, m, n, 5600 + n)
        check_pls(g, A, m, n, PAIR)


def test_pair_wide_stride_and_caller_workspace(g):
    """A row pitch above the minimum and a workspace of exactly gf2_workspace_bytes."""
    m, n = 1500, 1900
    st = S.default_stride(n) + 32
    A = make("dense", m, n, 5700, stride=st)
    R, P, Q, r = oracle.pls(A, m, n)
    need = g.workspace_bytes(g.OP_PLS, m, n, PAIR)
    work = torch.empty(need // 8 + 32, dtype=torch.int64, device="cuda")
    D = dev(A)
    Pd, Qd, rd = g.pls(D, n, work=work, opts=PAIR)
    torch.cuda.synchronize()
    assert int(rd.item()) == r
    assert (Pd.cpu().numpy() == P).all() and (Qd.cpu().numpy() == Q).all()
    W = S.words_per_row(n)
    assert (host(D)[:, :W] == R[:, :W]).all()
    assert (host(D)[:, W:] == A[:, W:]).all(), "words past the row's last word were written"


def test_pair_random_shapes_kinds_and_grids(g):
    """Seeded random shapes (1 .. 2600 rows and columns), input kinds and grid sizes, two panels
    per sweep, against the oracle."""
    rng = np.random.default_rng(20261204)
    for i in range(40):
        m = int(rng.integers(1, 2600))
        n = int(rng.integers(1, 2600))
        kind = KINDS[int(rng.integers(len(KINDS)))]
        grid = int(rng.choice([0, 2, 6, 37, 150]))
        A = make(kind, m, n, 7000 + i)
        opts = dict(PAIR, grid_ctas=grid) if grid else PAIR
        check_pls(g, A, m, n, opts)
