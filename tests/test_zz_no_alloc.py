"""The allocation-free rank entry point against the oracle and gf2_rank.

gf2_rank_noalloc serves callers that cannot call cudaMalloc: a plug-in whose
host application owns the whole device-memory budget, a latency-bound loop
that cannot take the device-wide synchronisation an allocation may bring, a
process whose device memory is already reserved by another framework's caching
allocator. It must return exactly the rank of the oracle (and of gf2_rank) on
consecutive calls that share its fixed scratch array, leave A untouched,
neither allocate device memory nor capture or replay a library graph, and
refuse matrices larger than the array. This file is collected last so that a
failure here never hides the other tests; it also passes alone in a fresh
process.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1006_1744_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GF2_ETOOBIG = 7


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_1744_gb300 import build, gf2
    build.build()
    return gf2.lib()


def _rank_via(lib, fn_name, A, n, out):
    m, stride = A.shape[0], A.stride(0)
    out.fill_(-1)
    s = torch.cuda.current_stream().cuda_stream
    if fn_name == "gf2_rank_noalloc":
        rc = lib.gf2_rank_noalloc(A.data_ptr(), m, n, stride, out.data_ptr(), s)
    else:
        rc = lib.gf2_rank(A.data_ptr(), m, n, stride, out.data_ptr(), None, 0, None, s)
    assert rc == 0, lib.gf2_strerror(rc)
    torch.cuda.synchronize()
    return int(out.item())


CASES = [
    ("dense", 1500, 1300, 11),      # nearly full rank, many panels
    ("sparse01", 900, 2000, 12),    # sparse, rank deficient
    ("lowrank", 700, 900, 14),      # rank 350 exactly
    ("dense", 4096, 4096, 13),      # the largest square that fits the array
]


@pytest.mark.parametrize("kind,m,n,seed", CASES)
def test_rank_noalloc_matches_oracle_on_consecutive_calls(kind, m, n, seed):
    lib = _lib()
    from paper_1006_1744_gb300 import gf2
    from tests.inputs import make
    A_np = make(kind, m, n, seed)
    want = oracle.rank(A_np, m, n)
    A = torch.from_numpy(A_np.view(np.int64)).cuda()
    before = A.clone()
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    assert _rank_via(lib, "gf2_rank", A, n, out) == want
    captured0, replayed0 = gf2.replay_stats()
    got1 = _rank_via(lib, "gf2_rank_noalloc", A, n, out)
    got2 = _rank_via(lib, "gf2_rank_noalloc", A, n, out)   # the same arguments again: no replay
    assert (got1, got2) == (want, want), (kind, m, n, want, got1, got2)
    assert gf2.replay_stats() == (captured0, replayed0)
    assert torch.equal(A, before)                           # input untouched


def test_rank_noalloc_steady_state_allocates_nothing():
    lib = _lib()
    n = m = 2048
    A_np = S.dense(m, n, 21)
    want = oracle.rank(A_np, m, n)
    A = torch.from_numpy(A_np.view(np.int64)).cuda()
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    assert _rank_via(lib, "gf2_rank_noalloc", A, n, out) == want   # warm-up: set-up and module loading
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _rank_via(lib, "gf2_rank_noalloc", A, n, out) == want
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_rank_noalloc_refuses_oversized_input():
    lib = _lib()
    n = 8192
    A = torch.zeros((8192, S.default_stride(n)), dtype=torch.int64, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.gf2_rank_noalloc(A.data_ptr(), 8192, n, A.stride(0), out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert rc == GF2_ETOOBIG
    assert b"scratch" in lib.gf2_strerror(rc)
