"""Thin ctypes binding of the C ABI in ``include/gf2.h`` (argument marshalling only).

Matrices are ``torch.int64`` CUDA tensors of shape (m, stride) holding the
packed bits (column j = bit j&63 of word j>>6); the bit patterns are those of
uint64. P, Q, rank and pivots are ``torch.int64`` CUDA tensors. Every call is
asynchronous on ``stream`` (default: PyTorch's current stream) and raises
``Gf2Error`` on a non-zero return code. There is no CPU fallback: a missing
``libgf2.so`` raises immediately.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libgf2.so")
_lock = threading.Lock()
_lib = None

OP_PLS, OP_RREF, OP_RANK, OP_MUL = 1, 2, 3, 4
PRODUCT_AUTO, PRODUCT_XOR, PRODUCT_TENSOR, PRODUCT_STRASSEN, PRODUCT_STRASSEN_TENSOR = 0, 1, 2, 3, 4
RREF_AUTO, RREF_PLS, RREF_M4RI, RREF_HYBRID = 0, 1, 2, 3
BATCH_AUTO, BATCH_STEPS, BATCH_PERSISTENT = 0, 1, 2

_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_int = ctypes.c_int


class Gf2Error(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = lib().gf2_strerror(code).decode()
        if code == 4:
            msg += f" (cudaError {lib().gf2_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [code {code}]")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("k", _int), ("tile_words", _int), ("grid_ctas", _int), ("product", _int),
                ("cutoff_cols", _i64), ("rref_method", _int), ("hybrid_permille", _int), ("batch_mode", _int),
                ("panels_per_sweep", _int), ("reserved", _int * 4)]


class BatchItem(ctypes.Structure):
    _fields_ = [("A", _vp), ("m", _i64), ("n", _i64), ("stride", _i64), ("P", _vp), ("Q", _vp)]


SYMBOLS = {
    "gf2_workspace_bytes": (_sz, [_int, _i64, _i64, _vp]),
    "gf2_mul_workspace_bytes": (_sz, [_i64, _i64, _i64, _vp]),
    "gf2_pls": (_int, [_vp, _i64, _i64, _i64, _vp, _vp, _vp, _vp, _sz, _vp, _vp]),
    "gf2_rref": (_int, [_vp, _i64, _i64, _i64, _vp, _vp, _vp, _sz, _vp, _vp]),
    "gf2_rank": (_int, [_vp, _i64, _i64, _i64, _vp, _vp, _sz, _vp, _vp]),
    "gf2_mul": (_int, [_vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64, _i64, _int, _vp, _sz, _vp, _vp]),
    "gf2_strerror": (ctypes.c_char_p, [_int]),
    "gf2_last_cuda_error": (_int, []),
    "gf2_version": (_int, []),
    "gf2_rank_noalloc": (_int, [_vp, _i64, _i64, _i64, _vp, _vp]),
    "gf2_pls_batched_workspace_bytes": (_sz, [_vp, _i64, _vp]),
    "gf2_pls_batched": (_int, [_vp, _i64, _vp, _vp, _sz, _vp, _vp]),
    "gf2_batch_plan": (_int, [_vp, _i64, _int, _vp, _vp, _vp]),
    "gf2_autotune": (_int, [_int, _i64, _i64, ctypes.c_double, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_double), _vp]),
    "gf2_sync_status": (_int, [_vp]),
    "gf2_diag_wait_timeout": (_int, [ctypes.c_uint64, _vp]),
    "gf2_replay_enable": (None, [_int]),
    "gf2_replay_stats": (None, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "gf2_prof_enable": (None, [_int]),
    "gf2_prof_reset": (None, []),
    "gf2_prof_launches": (ctypes.c_longlong, []),
    "gf2_prof_collect": (_int, [_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
}

PROF_SWEEP, PROF_PIVOT, PROF_RREF, PROF_MUL, PROF_COORDS = 0, 1, 2, 3, 4


def replay_enable(on: bool) -> None:
    """Switch graph replay of repeated pls/rref/rank calls on or off (process-wide)."""
    lib().gf2_replay_enable(1 if on else 0)


def replay_stats():
    """(graphs captured, calls replayed) since the process started."""
    c = ctypes.c_longlong(0)
    r = ctypes.c_longlong(0)
    lib().gf2_replay_stats(ctypes.byref(c), ctypes.byref(r))
    return int(c.value), int(r.value)


def prof_enable(flags: int) -> None:
    lib().gf2_prof_enable(flags)


def prof_reset() -> None:
    lib().gf2_prof_reset()


def prof_launches() -> int:
    return int(lib().gf2_prof_launches())


def prof_collect(cls: int):
    """(total milliseconds, launches) of one kernel class since prof_reset()."""
    ms = ctypes.c_double(0)
    n = ctypes.c_longlong(0)
    _check(lib().gf2_prof_collect(cls, ctypes.byref(ms), ctypes.byref(n)), "gf2_prof_collect")
    return ms.value, int(n.value)


def lib_path() -> str:
    return _LIBPATH


def lib():
    """Load libgf2.so (built by ``paper_1006_1744_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIBPATH):
                raise RuntimeError(f"{_LIBPATH} is missing: build it with `python -m paper_1006_1744_gb300.build` "
                                   "(there is no CPU fallback)")
            L = ctypes.CDLL(_LIBPATH)
            for name, (res, args) in SYMBOLS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _opts(opts):
    if opts is None:
        return None
    if isinstance(opts, Opts):
        return ctypes.byref(opts)
    o = Opts()
    for k, v in dict(opts).items():
        setattr(o, k, v)
    return ctypes.byref(o)


def _check(code, what):
    if code != 0:
        raise Gf2Error(code, what)


def _mat(A, n, what):
    if A.dtype != torch.int64 or A.dim() != 2 or not A.is_cuda:
        raise ValueError(f"{what}: expected a 2-D torch.int64 CUDA tensor (packed rows)")
    if A.numel() == 0:
        return A.shape[0], max(int(A.shape[1]), 16)
    if A.stride(1) != 1:
        raise ValueError(f"{what}: rows must be contiguous")
    return A.shape[0], A.stride(0)


def workspace_bytes(op: int, m: int, n: int, opts=None) -> int:
    return int(lib().gf2_workspace_bytes(op, m, n, _opts(opts)))


def new_workspace(op: int, m: int, n: int, device=None, opts=None) -> torch.Tensor:
    nbytes = workspace_bytes(op, m, n, opts)
    return torch.empty(max(nbytes, 256) // 8 + 32, dtype=torch.int64, device=device or "cuda")


def _work(work):
    if work is None:
        return None, 0
    base = work.data_ptr()
    aligned = (base + 255) // 256 * 256
    return aligned, work.numel() * 8 - (aligned - base)


def pls(A: torch.Tensor, n: int, P=None, Q=None, rank=None, work=None, opts=None, stream=None):
    """In-place PLS decomposition. Returns (P, Q, rank) device tensors."""
    m, stride = _mat(A, n, "gf2_pls")
    dev = A.device
    P = torch.empty(max(m, 1), dtype=torch.int64, device=dev) if P is None else P
    Q = torch.empty(max(n, 1), dtype=torch.int64, device=dev) if Q is None else Q
    rank = torch.empty(1, dtype=torch.int64, device=dev) if rank is None else rank
    wp, wb = _work(work)
    _check(lib().gf2_pls(_ptr(A), m, n, stride, _ptr(P), _ptr(Q), _ptr(rank), wp, wb, _opts(opts),
                         _stream(stream)), "gf2_pls")
    return P[:m], Q[:n], rank


def rref(A: torch.Tensor, n: int, rank=None, pivots=None, work=None, opts=None, stream=None,
         want_pivots=True):
    """In-place reduced row echelon form. Returns (rank, pivots) device tensors."""
    m, stride = _mat(A, n, "gf2_rref")
    dev = A.device
    rank = torch.empty(1, dtype=torch.int64, device=dev) if rank is None else rank
    if pivots is None and want_pivots:
        pivots = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    wp, wb = _work(work)
    _check(lib().gf2_rref(_ptr(A), m, n, stride, _ptr(rank), _ptr(pivots), wp, wb, _opts(opts),
                          _stream(stream)), "gf2_rref")
    return rank, (pivots[:n] if pivots is not None else None)


def rank(A: torch.Tensor, n: int, rank=None, work=None, opts=None, stream=None):
    """Rank (A unchanged). Returns a device tensor of shape (1,)."""
    m, stride = _mat(A, n, "gf2_rank")
    rank = torch.empty(1, dtype=torch.int64, device=A.device) if rank is None else rank
    wp, wb = _work(work)
    _check(lib().gf2_rank(_ptr(A), m, n, stride, _ptr(rank), wp, wb, _opts(opts), _stream(stream)),
           "gf2_rank")
    return rank


def rank_noalloc(A: torch.Tensor, n: int, rank=None, stream=None):
    """Rank using the library's fixed scratch array instead of any allocation."""
    m, stride = _mat(A, n, "gf2_rank_noalloc")
    rank = torch.empty(1, dtype=torch.int64, device=A.device) if rank is None else rank
    _check(lib().gf2_rank_noalloc(_ptr(A), m, n, stride, _ptr(rank), _stream(stream)), "gf2_rank_noalloc")
    return rank


def mul_workspace_bytes(m: int, k: int, n: int, opts=None) -> int:
    """Workspace bytes of mul() for A m x k and B k x n under opts (0 = none needed)."""
    return int(lib().gf2_mul_workspace_bytes(m, k, n, _opts(opts)))


def mul(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, m: int, k: int, n: int, accumulate=False,
        work=None, opts=None, stream=None):
    """C = A.B (or C + A.B) over GF(2), in place in C."""
    _, sc = _mat(C, n, "gf2_mul C")
    _, sa = _mat(A, k, "gf2_mul A")
    _, sb = _mat(B, n, "gf2_mul B")
    wp, wb = _work(work)
    _check(lib().gf2_mul(_ptr(C), sc, _ptr(A), sa, _ptr(B), sb, m, k, n, int(bool(accumulate)), wp, wb,
                         _opts(opts), _stream(stream)), "gf2_mul")
    return C


def sync_status(stream=None) -> int:
    """Waits for the stream; returns and clears the device status word (0 = ok)."""
    return int(lib().gf2_sync_status(_stream(stream)))


def diag_wait_timeout(limit_ns: int, stream=None) -> None:
    """Launches a kernel whose bounded wait on a never-set flag runs out."""
    _check(lib().gf2_diag_wait_timeout(int(limit_ns), _stream(stream)), "gf2_diag_wait_timeout")


def batch_items(mats, ns, Ps, Qs):
    """Host array of gf2_batch_item for device tensors (A_i of shape (m_i, stride_i))."""
    arr = (BatchItem * max(1, len(mats)))()
    for i, (A, n, P, Q) in enumerate(zip(mats, ns, Ps, Qs)):
        m, stride = _mat(A, n, "gf2_pls_batched")
        arr[i] = BatchItem(_ptr(A), m, n, stride, _ptr(P), _ptr(Q))
    return arr


def pls_batched_workspace_bytes(shapes, opts=None) -> int:
    """Workspace bytes for matrices of the given (m, n, stride) shapes."""
    items = (BatchItem * max(1, len(shapes)))()
    for i, (m, n, stride) in enumerate(shapes):
        items[i] = BatchItem(None, m, n, stride, None, None)
    return int(lib().gf2_pls_batched_workspace_bytes(items, len(shapes), _opts(opts)))


def batch_plan(shapes, ctas: int):
    """Host-only plan of the persistent batched schedule for (m, n) shapes on `ctas` CTAs.
    Returns (team_of per CTA, team sizes, team per matrix); -1 marks queue CTAs / queued matrices."""
    items = (BatchItem * max(1, len(shapes)))()
    for i, (m, n) in enumerate(shapes):
        items[i] = BatchItem(None, m, n, max(16, ((n + 63) // 64 + 15) // 16 * 16), None, None)
    team_of = (ctypes.c_int * max(1, ctas))()
    team_size = (ctypes.c_int * max(1, ctas))()
    member = (ctypes.c_int * max(1, len(shapes)))()
    nt = lib().gf2_batch_plan(items, len(shapes), ctas, team_of, team_size, member)
    if nt < 0:
        raise Gf2Error(1, "gf2_batch_plan")
    return list(team_of)[:ctas], list(team_size)[:nt], list(member)[:len(shapes)]


def pls_batched(mats, ns, Ps=None, Qs=None, ranks=None, work=None, opts=None, stream=None):
    """PLS of every matrix in `mats` (in place) in one batched call.
    Returns (Ps, Qs, ranks) with ranks a device int64 tensor of length len(mats)."""
    dev = mats[0].device if mats else torch.device("cuda")
    if Ps is None:
        Ps = [torch.empty(max(1, int(A.shape[0])), dtype=torch.int64, device=dev) for A in mats]
    if Qs is None:
        Qs = [torch.empty(max(1, int(n)), dtype=torch.int64, device=dev) for n in ns]
    ranks = torch.empty(max(1, len(mats)), dtype=torch.int64, device=dev) if ranks is None else ranks
    items = batch_items(mats, ns, Ps, Qs)
    wp, wb = _work(work)
    _check(lib().gf2_pls_batched(items, len(mats), _ptr(ranks), wp, wb, _opts(opts), _stream(stream)),
           "gf2_pls_batched")
    return Ps, Qs, ranks


def autotune(op: int, m: int, n: int, density: float = 0.5, stream=None):
    """Fastest gf2_opts for op on an m x n matrix of the given density (cached per size bucket).
    Returns (opts as a dict, mean milliseconds)."""
    best = Opts()
    ms = ctypes.c_double(0.0)
    _check(lib().gf2_autotune(op, m, n, float(density), ctypes.byref(best), ctypes.byref(ms), _stream(stream)),
           "gf2_autotune")
    return {"k": best.k, "tile_words": best.tile_words, "cutoff_cols": best.cutoff_cols, "product": best.product,
            "rref_method": best.rref_method, "hybrid_permille": best.hybrid_permille,
            "panels_per_sweep": best.panels_per_sweep}, ms.value
