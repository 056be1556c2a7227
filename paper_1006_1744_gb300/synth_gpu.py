"""Binding of the device twin of the seeded generators (``include/gf2_synth.h``).

Fills torch.int64 CUDA tensors with exactly the bits ``synth.py`` produces
(``dense`` for p == 0.5 without staircase, the per-bit recipe otherwise).
Holds none of the method's arithmetic.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_PATH = os.path.join(_HERE, "libgf2synth.so")
_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_PATH):
            raise RuntimeError(f"{_PATH} is missing: run `python -m paper_1006_1744_gb300.build`")
        L = ctypes.CDLL(_PATH)
        L.gf2_synth_fill.restype = ctypes.c_int
        L.gf2_synth_fill.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                     ctypes.c_uint64, ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        _lib = L
    return _lib


def fill(A: torch.Tensor, n: int, seed: int, p: float = 0.5, echelon_frac: float = 0.0, stream=None):
    assert A.dtype == torch.int64 and A.is_cuda and A.dim() == 2 and A.stride(1) == 1
    s = torch.cuda.current_stream().cuda_stream if stream is None else stream
    rc = lib().gf2_synth_fill(A.data_ptr(), A.shape[0], n, A.stride(0), seed & (2**64 - 1), p, echelon_frac, s)
    if rc:
        raise RuntimeError(f"gf2_synth_fill failed with code {rc}")
    return A


def dense(m: int, n: int, seed: int, stride: int | None = None, device="cuda") -> torch.Tensor:
    from .synth import default_stride
    stride = default_stride(n) if stride is None else stride
    A = torch.empty((m, stride), dtype=torch.int64, device=device)
    return fill(A, n, seed)
