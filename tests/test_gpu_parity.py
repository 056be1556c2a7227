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


@pytest.mark.parametrize("tile", [4, 8, 16])
def test_pls_parity_tile_and_grid_choices(g, tile):
    for grid in (1, 3, 152, 400):
        A = make("sparse05", 600, 900, grid)
        check_pls(g, A, 600, 900, opts={"tile_words": tile, "grid_ctas": grid})


@pytest.mark.parametrize("kind", KINDS)
def test_k4_tables_parity(g, kind):
    """Four-bit Gray-code tables (k = 4: sixteen tables of 16 entries per sweep) give
    the same PLS, rank and RREF (PLS route) as the oracle, alone and batched."""
    o = {"k": 4}
    for i, (m, n) in enumerate([(1, 1), (65, 65), (129, 300), (700, 500), (1024, 1024), (1300, 2100)]):
        A = make(kind, m, n, 4100 + i)
        check_pls(g, A, m, n, opts=o)
        D = dev(A)
        assert int(g.rank(D, n, opts=o).item()) == oracle.rank(A, m, n)
        R, piv, r = oracle.rref(A, m, n)
        rd, pd = g.rref(D, n, opts=o)
        torch.cuda.synchronize()
        W = S.words_per_row(n)
        assert int(rd.item()) == r and (pd.cpu().numpy()[:r] == piv).all()
        assert (host(D)[:, :W] == R[:, :W]).all()
    hosts = [(make(kind, m, n, 4200 + i), m, n) for i, (m, n) in enumerate([(300, 200), (129, 700), (2000, 300)])]
    ds = [dev(A) for (A, _, _) in hosts]
    Ps, Qs, ranks = g.pls_batched(ds, [n for (_, _, n) in hosts], opts={"k": 4, "batch_mode": g.BATCH_STEPS})
    torch.cuda.synchronize()
    for i, (A, m, n) in enumerate(hosts):
        R, P, Q, r = oracle.pls(A, m, n)
        assert int(ranks[i].item()) == r
        assert (Ps[i].cpu().numpy()[:m] == P[:m]).all() and (Qs[i].cpu().numpy()[:n] == Q[:n]).all()
        assert (host(ds[i])[:, :S.words_per_row(n)] == R[:, :S.words_per_row(n)]).all()


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


def test_repeated_calls_replay_with_new_contents(g):
    """The same argument list called again is replayed from a captured graph;
    every call, direct or replayed, must see the buffers' current contents."""
    g.replay_enable(True)
    m, n = 700, 900
    D = torch.empty((m, 32), dtype=torch.int64, device="cuda")  # stride 32 words > 15 used
    P = torch.empty(m, dtype=torch.int64, device="cuda")
    Q = torch.empty(n, dtype=torch.int64, device="cuda")
    rk = torch.empty(1, dtype=torch.int64, device="cuda")
    piv = torch.empty(n, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    c0, r0 = g.replay_stats()
    for it in range(6):
        kind = KINDS[it % len(KINDS)]
        A = make(kind, m, n, 900 + it)
        W = S.words_per_row(n)
        # PLS on the default stream
        D.zero_()
        D[:, :W].copy_(torch.from_numpy(np.ascontiguousarray(A[:, :W]).view(np.int64)))
        g.pls(D, n, P=P, Q=Q, rank=rk)
        torch.cuda.synchronize()
        R, Po, Qo, r = oracle.pls(A, m, n)
        assert int(rk.item()) == r and (P.cpu().numpy() == Po).all() and (Q.cpu().numpy() == Qo).all()
        assert (host(D)[:, :W] == R[:, :W]).all()
        # rank (input untouched) and RREF on another stream
        D[:, :W].copy_(torch.from_numpy(np.ascontiguousarray(A[:, :W]).view(np.int64)))
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            g.rank(D, n, rank=rk, stream=side)
        side.synchronize()
        assert int(rk.item()) == r
        with torch.cuda.stream(side):
            g.rref(D, n, rank=rk, pivots=piv, stream=side)
        side.synchronize()
        Rr, pv, rr = oracle.rref(A, m, n)
        assert int(rk.item()) == rr and (piv.cpu().numpy()[:rr] == pv).all()
        assert (host(D)[:, :W] == Rr[:, :W]).all()
    c1, r1 = g.replay_stats()
    assert c1 - c0 >= 3 and r1 - r0 >= 3 * 3, (c1 - c0, r1 - r0)


def test_replay_cache_eviction(g):
    """More distinct argument lists than the graph cache holds (32): each is run,
    captured and replayed, older graphs are dropped, and calls whose graph was
    dropped start over; every result matches the oracle."""
    g.replay_enable(True)
    m, n = 96, 130
    W = S.words_per_row(n)
    bufs = [(torch.empty((m, S.default_stride(n)), dtype=torch.int64, device="cuda"),
             torch.empty(m, dtype=torch.int64, device="cuda"), torch.empty(n, dtype=torch.int64, device="cuda"),
             torch.empty(1, dtype=torch.int64, device="cuda")) for _ in range(40)]
    work = g.new_workspace(g.OP_PLS, m, n)

    def run(i, seed):
        D, P, Q, rk = bufs[i]
        A = make("dense" if seed % 2 else "lowrank", m, n, seed)
        D.copy_(torch.from_numpy(np.ascontiguousarray(A).view(np.int64)))
        g.pls(D, n, P=P, Q=Q, rank=rk, work=work)
        torch.cuda.synchronize()
        R, Po, Qo, r = oracle.pls(A, m, n)
        assert int(rk.item()) == r and (P.cpu().numpy() == Po).all() and (Q.cpu().numpy() == Qo).all(), (i, seed)
        assert (host(D)[:, :W] == R[:, :W]).all(), (i, seed)

    c0, r0 = g.replay_stats()
    for i in range(40):
        for k in range(3):
            run(i, 1000 * i + k)
    for i in range(5):  # dropped long ago: direct, captured, replayed again
        for k in range(3):
            run(i, 7 + 1000 * i + k)
    c1, r1 = g.replay_stats()
    assert c1 - c0 == 45 and r1 - r0 == 45, (c1 - c0, r1 - r0)


def test_replay_off_matches(g):
    m, n = 300, 500
    A = S.dense(m, n, 77)
    g.replay_enable(False)
    try:
        c0, r0 = g.replay_stats()
        for _ in range(3):
            check_pls(g, A, m, n)
        assert g.replay_stats() == (c0, r0)
    finally:
        g.replay_enable(True)


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


def test_rref_and_rank_parity_wide_stride(g):
    """Row pitch above the minimum: the result must land in the caller's rows."""
    for (m, n, stride) in [(700, 900, 32), (300, 500, 48), (129, 64, 32)]:
        for kind in ("dense", "lowrank"):
            A = make(kind, m, n, 3 * m + stride)
            W = S.words_per_row(n)
            Aw = np.zeros((m, stride), dtype=np.uint64)
            Aw[:, :W] = A[:, :W]
            Aw[:, W:] = np.uint64(0x5A5A5A5A5A5A5A5A)  # words past the row must stay untouched
            D = dev(Aw)
            assert int(g.rank(D, n).item()) == oracle.rank(A, m, n)
            R, piv, r = oracle.rref(A, m, n)
            rd, pd = g.rref(D, n)
            torch.cuda.synchronize()
            assert int(rd.item()) == r and (pd.cpu().numpy()[:r] == piv).all()
            got = host(D)
            assert (got[:, :W] == R[:, :W]).all()
            assert (got[:, W:] == np.uint64(0x5A5A5A5A5A5A5A5A)).all()


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


@pytest.mark.parametrize("product", [3, 4])
@pytest.mark.parametrize("acc", [False, True])
def test_mul_strassen_parity(g, product, acc):
    """Strassen-Winograd products (XOR-table and tensor-core leaves) equal the
    plain product bit for bit: leaf size 512 gives up to two levels here (a
    level needs k and n multiples of 2048), and shapes that do not split fall
    back to the leaf form."""
    rng = np.random.default_rng(11 + product + 2 * acc)
    opts = {"product": product, "cutoff_cols": 512}
    for (m, k, n) in [(2048, 2048, 2048), (4096, 2048, 4096), (2048, 4096, 2048), (4096, 4096, 4096),
                      (1000, 2048, 2048), (2048, 3000, 2048), (1024, 1024, 1024)]:
        A = S.dense(m, k, int(rng.integers(1 << 30)))
        B = S.dense(k, n, int(rng.integers(1 << 30)))
        C0 = S.dense(m, n, int(rng.integers(1 << 30)))
        want = oracle.mul(A, B, m, k, n, C=C0 if acc else None, stride=C0.shape[1])
        Cd = dev(C0)
        nb = g.mul_workspace_bytes(m, k, n, opts)
        work = torch.empty(max(nb // 8, 1) + 32, dtype=torch.int64, device="cuda")
        g.mul(Cd, dev(A), dev(B), m, k, n, accumulate=acc, work=work, opts=opts)
        torch.cuda.synchronize()
        W = S.words_per_row(n)
        assert (host(Cd)[:, :W] == want[:, :W]).all(), (m, k, n)


def test_mul_strassen_three_levels_and_wide_strides(g):
    """Three Strassen-Winograd levels (8192 -> 4096 -> 2048 -> 1024-bit leaves, leaf
    size 512), and every block view formed from row pitches wider than the
    minimum (A, B and C each 16, 32 and 48 words wider): both leaf forms, with and
    without accumulation, equal the oracle's product; C's padding words stay."""
    m = k = n = 8192
    A = S.dense(m, k, 71)
    B = S.dense(k, n, 72)
    C0 = S.dense(m, n, 73)
    want = {False: oracle.mul(A, B, m, k, n, stride=C0.shape[1]), True: oracle.mul(A, B, m, k, n, C=C0)}
    for product in (3, 4):
        for acc in (False, True):
            opts = {"product": product, "cutoff_cols": 512}
            Cd = dev(C0)
            g.mul(Cd, dev(A), dev(B), m, k, n, accumulate=acc, opts=opts)
            torch.cuda.synchronize()
            assert (host(Cd) == want[acc]).all(), (product, acc)
    m = k = n = 4096
    W = S.words_per_row(n)
    A = S.dense(m, k, 81)
    B = S.dense(k, n, 82)
    C0 = S.dense(m, n, 83)

    def wide(M, extra):
        out = np.full((M.shape[0], M.shape[1] + extra), np.uint64(0x5A5A5A5A5A5A5A5A), dtype=np.uint64)
        out[:, :W] = M[:, :W]
        return out

    want = {False: oracle.mul(A, B, m, k, n), True: oracle.mul(A, B, m, k, n, C=C0)}
    for product in (3, 4):
        for acc in (False, True):
            Cd = dev(wide(C0, 48))
            g.mul(Cd, dev(wide(A, 16)), dev(wide(B, 32)), m, k, n, accumulate=acc,
                  opts={"product": product, "cutoff_cols": 512})
            torch.cuda.synchronize()
            got = host(Cd)
            assert (got[:, :W] == want[acc][:, :W]).all(), ("wide", product, acc)
            assert (got[:, W:] == np.uint64(0x5A5A5A5A5A5A5A5A)).all()


def test_mul_strassen_internal_workspace_and_too_small(g):
    m = k = n = 4096
    opts = {"product": 3, "cutoff_cols": 1024}
    A = S.dense(m, k, 5)
    B = S.dense(k, n, 6)
    want = oracle.mul(A, B, m, k, n)
    Cd = torch.zeros((m, S.default_stride(n)), dtype=torch.int64, device="cuda")
    g.mul(Cd, dev(A), dev(B), m, k, n, opts=opts)  # internal workspace
    torch.cuda.synchronize()
    assert (host(Cd) == want).all()
    small = torch.empty(64, dtype=torch.int64, device="cuda")
    with pytest.raises(g.Gf2Error):
        g.mul(Cd, dev(A), dev(B), m, k, n, work=small, opts=opts)


def test_autotune_product_with_strassen_candidates(g):
    """At 16384^2 the product's candidates include both Strassen forms; whatever
    is chosen gives the same product as the XOR-table form."""
    from paper_1006_1744_gb300 import synth_gpu
    n = 16384
    om, ms = g.autotune(g.OP_MUL, n, n, 0.5)
    assert om["product"] in (1, 2, 3, 4) and ms > 0
    A = synth_gpu.dense(n, n, 21)
    B = synth_gpu.dense(n, n, 22)
    ref = torch.zeros_like(A)
    g.mul(ref, A, B, n, n, n, opts={"product": 1})
    C = torch.zeros_like(A)
    g.mul(C, A, B, n, n, n, opts=om)
    torch.cuda.synchronize()
    assert torch.equal(C, ref)


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


TC = {"product": 2}
MUL_SHAPES_TC = [(1, 1, 1), (64, 64, 64), (100, 130, 70), (513, 1000, 300), (1024, 1024, 1024),
                 (2000, 65, 129), (37, 3000, 515), (129, 8300, 257), (300, 16500, 600)]


@pytest.mark.parametrize("acc", [False, True])
def test_mul_tensor_parity(g, acc):
    """Tensor-core product (0/1 FP8 operands, FP32 sums, low bit) against the
    oracle's product; inner dimensions past one accumulation segment (8192 bits)."""
    rng = np.random.default_rng(11)
    for (m, k, n) in MUL_SHAPES_TC:
        A = S.dense(m, k, int(rng.integers(1 << 30)))
        B = S.dense(k, n, int(rng.integers(1 << 30)))
        C0 = S.dense(m, n, int(rng.integers(1 << 30)))
        want = oracle.mul(A, B, m, k, n, C=C0 if acc else None, stride=C0.shape[1])
        Cd = dev(C0)
        g.mul(Cd, dev(A), dev(B), m, k, n, accumulate=acc, opts=TC)
        torch.cuda.synchronize()
        W = S.words_per_row(n)
        assert (host(Cd)[:, :W] == want[:, :W]).all(), (m, k, n)
    assert g.sync_status() == 0


def test_mul_tensor_all_ones_sums(g):
    """All-ones operands: every sum equals the inner dimension, so the parity of
    each output bit is k mod 2 (the largest sums the accumulator sees)."""
    for k in (31, 8191, 8192, 8193, 16383):
        m, n = 130, 300
        A = S.pack(np.ones((m, k), dtype=bool))
        B = S.pack(np.ones((k, n), dtype=bool))
        C = torch.zeros((m, S.default_stride(n)), dtype=torch.int64, device="cuda")
        g.mul(C, dev(A), dev(B), m, k, n, opts=TC)
        torch.cuda.synchronize()
        want = S.pack(np.full((m, n), k & 1, dtype=bool))
        assert (host(C) == want).all(), k


def test_mul_tensor_views_with_foreign_bits(g):
    """A, B and C as views inside wider matrices (the recursive PLS's A_SW, A_NE
    and A_SE): bits of A past column k and of B past column n are other data and
    must not leak in; C's words past its last column are not written."""
    rng = np.random.default_rng(5)
    for (m, k, n) in [(200, 100, 150), (300, 700, 333), (129, 64, 65)]:
        Af = S.dense(m, k + 200, int(rng.integers(1 << 30)))
        Bf = S.dense(k + 50, n + 300, int(rng.integers(1 << 30)))
        Cf = S.dense(m, n + 300, int(rng.integers(1 << 30)))
        Ak = S.pack(S.unpack(Af, m, k + 200)[:, :k])
        Bk = S.pack(S.unpack(Bf, k + 50, n + 300)[:k, :n])
        Ck = S.pack(S.unpack(Cf, m, n + 300)[:, :n])
        want = S.unpack(oracle.mul(Ak, Bk, m, k, n, C=Ck, stride=Ck.shape[1]), m, n)
        Cd = dev(Cf)
        g.mul(Cd, dev(Af), dev(Bf)[:k], m, k, n, accumulate=True, opts=TC)
        torch.cuda.synchronize()
        got = S.unpack(host(Cd), m, n + 300)
        assert (got[:, :n] == want).all()
        assert (got[:, n:] == S.unpack(Cf, m, n + 300)[:, n:]).all()


@pytest.mark.parametrize("cutoff", [128, 256])
def test_recursive_pls_tensor_product_parity(g, cutoff):
    """Recursive PLS with the tensor-core trailing product: identical to the
    Gaussian PLS, like the XOR-table form."""
    for i, (m, n) in enumerate([(300, 1000), (1000, 700), (1500, 2000)]):
        for kind in ("dense", "lowrank", "sparse05", "echelon"):
            A = make(kind, m, n, 1700 + 13 * i + cutoff)
            check_pls(g, A, m, n, opts={"cutoff_cols": cutoff, "product": 2})
    assert g.sync_status() == 0


def test_bounded_wait_reports_timeout(g):
    """A wait on a flag nothing sets gives up after its limit and records
    GF2_ETIMEOUT; the context stays usable and the status clears on reading."""
    assert g.sync_status() == 0
    g.diag_wait_timeout(20_000_000)
    assert g.sync_status() == 8
    assert g.sync_status() == 0
    A = S.dense(100, 100, 3)
    check_pls(g, A, 100, 100)


def test_pls_batched_parity(g):
    """Batched PLS: every matrix of a mixed batch (shapes, densities, empty and
    degenerate members) matches the oracle exactly, like gf2_pls on it alone."""
    rng = np.random.default_rng(21)
    shapes = [(0, 0), (0, 70), (50, 0), (1, 1), (64, 64), (300, 200), (129, 700), (700, 129),
              (257, 257), (1000, 1500), (90, 64), (2000, 300)]
    kinds = ["dense", "sparse05", "sparse01", "echelon", "lowrank", "deep", "dup", "zero", "identity", "ones"]
    hosts, mats, ns = [], [], []
    for i, (m, n) in enumerate(shapes * 2):
        kind = kinds[i % len(kinds)]
        A = make(kind, m, n, int(rng.integers(1 << 30))) if m and n else np.zeros((m, S.default_stride(n)),
                                                                                  dtype=np.uint64)
        hosts.append((A, m, n))
        mats.append(dev(A))
        ns.append(n)
    for opts in (None, {"tile_words": 4}, {"batch_mode": g.BATCH_STEPS}, {"batch_mode": g.BATCH_PERSISTENT}):
        ds = [t.clone() for t in mats]
        Ps, Qs, ranks = g.pls_batched(ds, ns, opts=opts)
        torch.cuda.synchronize()
        rk = ranks.cpu().numpy()
        for i, (A, m, n) in enumerate(hosts):
            R, P, Q, r = oracle.pls(A, m, n)
            assert rk[i] == r, (i, m, n)
            assert (Ps[i].cpu().numpy()[:m] == P[:m]).all(), i
            assert (Qs[i].cpu().numpy()[:n] == Q[:n]).all(), i
            if m and n:
                W = S.words_per_row(n)
                assert (host(ds[i])[:, :W] == R[:, :W]).all(), (i, m, n)


@pytest.mark.parametrize("mode", [1, 2])
def test_pls_batched_many_small_and_user_workspace(g, mode):
    """A batch of 300 small matrices of varied shape through a caller-owned
    workspace, run twice (the workspace's previous contents do not matter), with
    both schedules (launches per panel step; one persistent launch)."""
    rng = np.random.default_rng(8)
    hosts, ns = [], []
    for i in range(300):
        m = int(rng.integers(1, 200))
        n = int(rng.integers(1, 300))
        p = [0.5, 0.1, 0.01][i % 3]
        hosts.append((S.bernoulli(m, n, p, 5000 + i), m, n))
        ns.append(n)
    shapes = [(m, n, S.default_stride(n)) for (_, m, n) in hosts]
    nbytes = g.pls_batched_workspace_bytes(shapes)
    work = torch.empty(nbytes // 8 + 64, dtype=torch.int64, device="cuda")
    want = [oracle.pls(A, m, n) for (A, m, n) in hosts]
    for _ in range(2):
        ds = [dev(A) for (A, _, _) in hosts]
        Ps, Qs, ranks = g.pls_batched(ds, ns, work=work, opts={"batch_mode": mode})
        torch.cuda.synchronize()
        rk = ranks.cpu().numpy()
        for i, (A, m, n) in enumerate(hosts):
            R, P, Q, r = want[i]
            assert rk[i] == r
            assert (Ps[i].cpu().numpy()[:m] == P[:m]).all()
            assert (Qs[i].cpu().numpy()[:n] == Q[:n]).all()
            assert (host(ds[i])[:, :S.words_per_row(n)] == R[:, :S.words_per_row(n)]).all()


@pytest.mark.parametrize("mode", [1, 2])
def test_pls_batched_replayed_with_new_contents(g, mode):
    """The same batch (buffers, ranks, workspace) called again is replayed from a
    captured graph, plan upload included; each call sees the current contents."""
    g.replay_enable(True)
    rng = np.random.default_rng(33)
    shapes = [(int(rng.integers(1, 400)), int(rng.integers(1, 500))) for _ in range(40)]
    mats = [torch.empty((m, S.default_stride(n)), dtype=torch.int64, device="cuda") for (m, n) in shapes]
    ns = [n for (_, n) in shapes]
    Ps = [torch.empty(m, dtype=torch.int64, device="cuda") for (m, _) in shapes]
    Qs = [torch.empty(n, dtype=torch.int64, device="cuda") for (_, n) in shapes]
    ranks = torch.empty(len(shapes), dtype=torch.int64, device="cuda")
    work = torch.empty(g.pls_batched_workspace_bytes([(m, n, S.default_stride(n)) for (m, n) in shapes]) // 8 + 64,
                       dtype=torch.int64, device="cuda")
    c0, r0 = g.replay_stats()
    kinds = ["dense", "sparse01", "lowrank", "echelon"]
    for it in range(5):
        hosts = [make(kinds[(i + it) % 4], m, n, 100 * it + i) for i, (m, n) in enumerate(shapes)]
        for D, A in zip(mats, hosts):
            D.copy_(torch.from_numpy(np.ascontiguousarray(A).view(np.int64)))
        g.pls_batched(mats, ns, Ps=Ps, Qs=Qs, ranks=ranks, work=work, opts={"batch_mode": mode})
        torch.cuda.synchronize()
        rk = ranks.cpu().numpy()
        for i, ((m, n), A) in enumerate(zip(shapes, hosts)):
            R, P, Q, r = oracle.pls(A, m, n)
            assert rk[i] == r, (it, i)
            assert (Ps[i].cpu().numpy() == P[:m]).all() and (Qs[i].cpu().numpy() == Q[:n]).all(), (it, i)
            W = S.words_per_row(n)
            assert (host(mats[i])[:, :W] == R[:, :W]).all(), (it, i)
    c1, r1 = g.replay_stats()
    assert c1 - c0 == 1 and r1 - r0 == 3, (c1 - c0, r1 - r0)


def test_pls_batched_persistent_teams(g):
    """A batch whose large members go to teams of several CTAs in the persistent
    launch (team barriers between pivot search and sweep), mixed with small ones:
    every member equals the oracle, as with the per-step schedule."""
    rng = np.random.default_rng(44)
    shapes = [(3000, 4000), (2500, 2500), (4096, 2048), (2000, 3000)] + \
             [(int(rng.integers(1, 300)), int(rng.integers(1, 400))) for _ in range(60)]
    kinds = ["dense", "sparse01", "lowrank", "echelon", "deep"]
    hosts = [(make(kinds[i % 5], m, n, 900 + i), m, n) for i, (m, n) in enumerate(shapes)]
    want = [oracle.pls(A, m, n) for (A, m, n) in hosts]
    for mode in (g.BATCH_PERSISTENT, g.BATCH_STEPS):
        ds = [dev(A) for (A, _, _) in hosts]
        Ps, Qs, ranks = g.pls_batched(ds, [n for (_, _, n) in hosts], opts={"batch_mode": mode})
        torch.cuda.synchronize()
        assert g.sync_status() == 0
        rk = ranks.cpu().numpy()
        for i, (A, m, n) in enumerate(hosts):
            R, P, Q, r = want[i]
            assert rk[i] == r, (mode, i)
            assert (Ps[i].cpu().numpy()[:m] == P[:m]).all() and (Qs[i].cpu().numpy()[:n] == Q[:n]).all(), (mode, i)
            W = S.words_per_row(n)
            assert (host(ds[i])[:, :W] == R[:, :W]).all(), (mode, i)


def test_pls_batched_persistent_many_medium_members(g):
    """160 members of 2048 to 2600 rows, enough that the persistent plan forms no team: each
    member is eliminated by one CTA from the work queue (the pivot search of panel b + 1 beside
    the sweep of panel b). Every input kind, word counts from one up, pivots past the window and
    rank deficiency, against the oracle."""
    rng = np.random.default_rng(61)
    kinds = ["dense", "sparse05", "sparse01", "echelon", "lowrank", "deep", "dup", "zero", "identity", "ones"]
    hosts = []
    for i in range(160):
        m = int(rng.integers(2048, 2600))
        n = int(rng.choice([1, 63, 64, 65, 128, 129, 192, 256, 300, 449, 640, 700]))
        hosts.append((make(kinds[i % len(kinds)], m, n, 6100 + i), m, n))
    team_of, team_size, member_team = g.batch_plan([(m, n) for (_, m, n) in hosts], 152)
    assert (np.asarray(member_team) < 0).all(), "a member went to a team"
    want = [oracle.pls(A, m, n) for (A, m, n) in hosts]
    ds = [dev(A) for (A, _, _) in hosts]
    Ps, Qs, ranks = g.pls_batched(ds, [n for (_, _, n) in hosts], opts={"batch_mode": g.BATCH_PERSISTENT})
    torch.cuda.synchronize()
    assert g.sync_status() == 0
    rk = ranks.cpu().numpy()
    for i, (A, m, n) in enumerate(hosts):
        R, P, Q, r = want[i]
        assert rk[i] == r, (i, m, n)
        assert (Ps[i].cpu().numpy()[:m] == P[:m]).all() and (Qs[i].cpu().numpy()[:n] == Q[:n]).all(), (i, m, n)
        W = S.words_per_row(n)
        assert (host(ds[i])[:, :W] == R[:, :W]).all(), (i, m, n)


def test_autotune_choices_are_exact_and_cached(g):
    """The autotuner only picks among settings that change no result: PLS with its
    choice matches the oracle, and a second call returns the cached choice."""
    m, n = 1500, 2100
    o1, ms1 = g.autotune(g.OP_PLS, m, n, 0.5)
    # a tile width of the one-panel sweep, or one or two panels per sweep at the default tiles
    assert (o1["tile_words"] in (4, 8, 16) or o1["panels_per_sweep"] in (1, 2)) and ms1 > 0
    o2, ms2 = g.autotune(g.OP_PLS, m, n, 0.5)
    assert (o1, ms1) == (o2, ms2)
    check_pls(g, S.dense(m, n, 77), m, n, opts=o1)
    om, _ = g.autotune(g.OP_MUL, 1024, 1024, 0.5)
    assert om["product"] in (1, 2)
    rng = np.random.default_rng(9)
    A = S.dense(300, 1024, int(rng.integers(1 << 30)))
    B = S.dense(1024, 700, int(rng.integers(1 << 30)))
    want = oracle.mul(A, B, 300, 1024, 700)
    C = torch.zeros((300, S.default_stride(700)), dtype=torch.int64, device="cuda")
    g.mul(C, dev(A), dev(B), 300, 1024, 700, opts=om)
    torch.cuda.synchronize()
    assert (host(C)[:, :11] == want[:, :11]).all()
    # RREF: the route (PLS, M4RI, hybrid) is among the candidates; the choice is exact
    for (mr, nr, dens) in [(1200, 1700, 0.5), (1500, 1500, 0.02)]:
        orr, _ = g.autotune(g.OP_RREF, mr, nr, dens)
        assert orr["rref_method"] in (0, 2, 3)
        A = S.bernoulli(mr, nr, dens, 123) if dens < 0.5 else S.dense(mr, nr, 123)
        R, piv, r = oracle.rref(A, mr, nr)
        D = dev(A)
        rd, pd = g.rref(D, nr, opts=orr)
        torch.cuda.synchronize()
        W = S.words_per_row(nr)
        assert int(rd.item()) == r and (pd.cpu().numpy()[:r] == piv).all()
        assert (host(D)[:, :W] == R[:, :W]).all()
    assert g.sync_status() == 0
