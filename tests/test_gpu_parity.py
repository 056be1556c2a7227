"""Bit-exact parity of the CUDA path (called through the C ABI) with the CPU
oracle on seeded inputs: rank, P, Q, the in-place PLS matrix, RREF, pivots,
the product, and the device generator. Sizes span several 64-column panels,
the 128-row pivot window and ragged tails; degenerate inputs included."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1006_1744_gb300 import synth as S

from tests.inputs import KINDS, make

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


SHAPES = [(1, 1), (1, 64), (64, 1), (7, 13), (64, 64), (65, 65), (100, 200), (200, 100), (128, 128),
          (129, 300), (257, 257), (300, 64), (500, 700), (700, 500), (1024, 1024)]


def check_pls(g, A, m, n, opts=None, work=None):
    R, P, Q, r = oracle.pls(A, m, n)
    D = dev(A)
    Pd, Qd, rd = g.pls(D, n, opts=opts, work=work)
    torch.cuda.synchronize()
    assert int(rd.item()) == r
    assert (Pd.cpu().numpy() == P).all(), "P differs"
    assert (Qd.cpu().numpy() == Q).all(), "Q differs"
    W = S.words_per_row(n)
    got = host(D)[:, :W]
    bad = np.nonzero((got != R[:, :W]).any(axis=1))[0]
    assert bad.size == 0, f"rows differ: {bad[:10]}"
    return r


@pytest.mark.parametrize("kind", KINDS)
def test_pls_parity_shapes(g, kind):
    for i, (m, n) in enumerate(SHAPES):
        A = make(kind, m, n, 100 + i)
        check_pls(g, A, m, n)


def test_pls_parity_config1_many_seeds(g):
    """1024 x 1024 dense Bernoulli(1/2), table width k = 8, many seeds."""
    for seed in range(1, 41):
        A = S.dense(1024, 1024, seed)
        check_pls(g, A, 1024, 1024, opts={"k": 8})


@pytest.mark.parametrize("tile", [4, 8])
def test_pls_parity_tile_and_grid_choices(g, tile):
    for grid in (1, 3, 152, 400):
        A = make("sparse05", 600, 900, grid)
        check_pls(g, A, 600, 900, opts={"tile_words": tile, "grid_ctas": grid})


def test_pls_parity_wide_stride_and_user_workspace(g):
    m, n = 300, 500
    A = S.dense(m, n, 5, stride=48)
    work = g.new_workspace(g.OP_PLS, m, n)
    for _ in range(2):
        check_pls(g, A, m, n, work=work)


def test_pls_parity_tall_and_wide(g):
    for (m, n) in [(3000, 200), (150, 4000), (2049, 2049)]:
        for kind in ("dense", "sparse01", "lowrank"):
            check_pls(g, make(kind, m, n, m + n), m, n)


def test_pls_empty(g):
    for (m, n) in [(0, 10), (10, 0), (0, 0)]:
        D = torch.zeros((max(m, 1), 16), dtype=torch.int64, device="cuda")[:m]
        P, Q, r = g.pls(D, n)
        torch.cuda.synchronize()
        assert int(r.item()) == 0
        assert (P.cpu().numpy() == np.arange(m)).all() and (Q.cpu().numpy() == np.arange(n)).all()


def check_rref(g, A, m, n):
    R, piv, r = oracle.rref(A, m, n)
    D = dev(A)
    rd, pd = g.rref(D, n)
    torch.cuda.synchronize()
    assert int(rd.item()) == r
    pv = pd.cpu().numpy()
    assert (pv[:r] == piv).all() and (pv[r:] == np.arange(r, n)).all()
    W = S.words_per_row(n)
    got = host(D)[:, :W]
    bad = np.nonzero((got != R[:, :W]).any(axis=1))[0]
    assert bad.size == 0, f"rows differ: {bad[:10]}"


@pytest.mark.parametrize("kind", KINDS)
def test_rref_parity_shapes(g, kind):
    for i, (m, n) in enumerate(SHAPES):
        check_rref(g, make(kind, m, n, 500 + i), m, n)


def test_rref_parity_wide_rank_deficient(g):
    for (m, n) in [(300, 2000), (1000, 1500), (2100, 700)]:
        for kind in ("dense", "lowrank", "echelon", "sparse01"):
            check_rref(g, make(kind, m, n, 7 * m + n), m, n)


def test_rank_parity_and_input_untouched(g):
    for kind in KINDS:
        for (m, n) in [(129, 300), (1024, 1024), (700, 500)]:
            A = make(kind, m, n, 31 + m)
            D = dev(A)
            r = g.rank(D, n)
            torch.cuda.synchronize()
            assert int(r.item()) == oracle.rank(A, m, n)
            assert (host(D) == A).all()


@pytest.mark.parametrize("acc", [False, True])
def test_mul_parity(g, acc):
    rng = np.random.default_rng(3)
    for (m, k, n) in [(1, 1, 1), (64, 64, 64), (100, 130, 70), (513, 1000, 300), (1024, 1024, 1024),
                      (2000, 65, 129), (37, 3000, 515)]:
        A = S.dense(m, k, int(rng.integers(1 << 30)))
        B = S.dense(k, n, int(rng.integers(1 << 30)))
        C0 = S.dense(m, n, int(rng.integers(1 << 30)))
        want = oracle.mul(A, B, m, k, n, C=C0 if acc else None, stride=C0.shape[1])
        Cd = dev(C0)
        g.mul(Cd, dev(A), dev(B), m, k, n, accumulate=acc)
        torch.cuda.synchronize()
        W = S.words_per_row(n)
        assert (host(Cd)[:, :W] == want[:, :W]).all()


def test_device_generator_matches_host(g):
    from paper_1006_1744_gb300 import synth_gpu
    for (m, n) in [(1, 1), (70, 130), (300, 64), (257, 1000)]:
        st = S.default_stride(n)
        D = torch.empty((m, st), dtype=torch.int64, device="cuda")
        synth_gpu.fill(D, n, 99)
        assert (host(D) == S.dense(m, n, 99)).all()
        synth_gpu.fill(D, n, 7, p=0.01)
        assert (host(D) == S.bernoulli(m, n, 0.01, 7)).all()
        synth_gpu.fill(D, n, 8, p=0.3, echelon_frac=0.5)
        assert (host(D) == S.echelon(m, n, 0.3, 8)).all()


@pytest.mark.parametrize("cutoff", [128, 256, 512])
def test_recursive_pls_parity(g, cutoff):
    """Recursive PLS (split, row gathers, lower solve, product, second call, merge)
    down to the panel elimination at the cutoff: identical to the Gaussian PLS."""
    shapes = [(300, 1000), (1000, 700), (640, 640), (257, 1300), (1500, 2000)]
    for i, (m, n) in enumerate(shapes):
        for kind in ("dense", "lowrank", "sparse05", "echelon", "deep", "zero"):
            A = make(kind, m, n, 900 + 13 * i + cutoff)
            check_pls(g, A, m, n, opts={"cutoff_cols": cutoff})


def test_recursive_pls_user_workspace(g):
    m, n = 1100, 1500
    opts = {"cutoff_cols": 256}
    work = g.new_workspace(g.OP_PLS, m, n, opts=opts)
    for seed in (1, 2):
        check_pls(g, S.dense(m, n, seed), m, n, opts=opts, work=work)
