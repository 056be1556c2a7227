"""The allocation-free rank entry point agrees with gf2_rank.

gf2_rank_noalloc serves callers that may not call cudaMalloc (code running
under CUDA graph capture, loops that cannot afford an allocation's device
stall, plug-ins whose host owns all device memory). It must return exactly the
rank gf2_rank returns, on consecutive calls that share its fixed scratch
array, and refuse matrices larger than that array. This file is collected last
so that a failure here never hides the other tests.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

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


def _rank_via(lib, fn_name, A, n):
    m, stride = A.shape[0], A.stride(0)
    out = torch.full((1,), -1, dtype=torch.int64, device=A.device)
    s = torch.cuda.current_stream().cuda_stream
    if fn_name == "gf2_rank_noalloc":
        rc = lib.gf2_rank_noalloc(A.data_ptr(), m, n, stride, out.data_ptr(), s)
    else:
        rc = lib.gf2_rank(A.data_ptr(), m, n, stride, out.data_ptr(), None, 0, None, s)
    assert rc == 0, lib.gf2_strerror(rc)
    torch.cuda.synchronize()
    return int(out.item())


def test_rank_noalloc_matches_rank_on_consecutive_calls():
    lib = _lib()
    cases = [
        (S.dense(1500, 1300, 11), 1500, 1300),                       # full rank-ish, many panels
        (S.bernoulli(900, 2000, 0.01, 12), 900, 2000),               # sparse, rank deficient
        (S.dense(4096, 4096, 13), 4096, 4096),                       # largest square that fits
    ]
    for A_np, m, n in cases:
        A = torch.from_numpy(A_np.view(np.int64)).cuda()
        before = A.clone()
        want = _rank_via(lib, "gf2_rank", A, n)
        got1 = _rank_via(lib, "gf2_rank_noalloc", A, n)
        got2 = _rank_via(lib, "gf2_rank_noalloc", A, n)   # second call reuses the same scratch
        assert got1 == want and got2 == want, (m, n, want, got1, got2)
        assert torch.equal(A, before)                       # input untouched


def test_rank_noalloc_refuses_oversized_input():
    lib = _lib()
    n = 8192
    A = torch.zeros((8192, S.default_stride(n)), dtype=torch.int64, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.gf2_rank_noalloc(A.data_ptr(), 8192, n, A.stride(0), out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert rc == GF2_ETOOBIG
    assert b"scratch" in lib.gf2_strerror(rc)
