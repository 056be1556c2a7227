"""Seeded synthetic GF(2) matrices (numpy, host side).

This module holds only the counter-based input generators. It contains none of
the elimination, table or product arithmetic; both the CPU oracle and the CUDA
path receive their inputs from here (the CUDA twin in ``csrc/synth.cu``
implements the same published SplitMix64 mixer so that large inputs can be
filled on the device, and tests check the two bit for bit).

Layout produced: row-major packed uint64 words, column ``j`` in word ``j >> 6``
at bit ``j & 63`` (least significant bit = leftmost column). ``stride`` is the
row pitch in words; padding bits (columns >= n) and padding words are zero.

Generators (all inputs are 64-bit counters, so any element can be produced
independently of the others):

* ``mix(x)``: the SplitMix64 output function (Steele, Lea, Flood, "Fast
  splittable pseudorandom number generators", OOPSLA 2014), i.e. add the golden
  gamma 0x9E3779B97F4A7C15 then apply the 30/27/31 xor-shift-multiply finalizer.
* dense Bernoulli(1/2): ``word(i, w) = mix(seed ^ mix((i << 32) | w))``.
* Bernoulli(p): ``bit(i, j) = (mix(seed ^ TAG_P ^ mix((i << 32) | j)) >> 11)
  < floor(p * 2**53)``.
* echelon-structured (staircase): row ``i`` is zero before column
  ``floor(frac * i * n / m)`` and Bernoulli(p) from there on.
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
MUL1 = np.uint64(0xBF58476D1CE4E5B9)
MUL2 = np.uint64(0x94D049BB133111EB)
TAG_P = np.uint64(0xD1B54A32D192ED03)
HEADLINE_SEED = 0x10061744

_U64 = np.uint64


def mix(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 ``x``."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + GOLDEN_GAMMA).astype(np.uint64)
        z = (z ^ (z >> _U64(30))) * MUL1
        z = (z ^ (z >> _U64(27))) * MUL2
        return z ^ (z >> _U64(31))


def words_per_row(n: int) -> int:
    return (n + 63) // 64


def default_stride(n: int) -> int:
    """Row pitch in words: a multiple of 16 words (128 bytes), at least 16."""
    w = words_per_row(n)
    return max(16, (w + 15) // 16 * 16)


def _pad_mask(n: int, stride: int) -> np.ndarray:
    """Per-word mask that keeps columns < n and clears padding bits/words."""
    mask = np.zeros(stride, dtype=np.uint64)
    full, rem = divmod(n, 64)
    mask[:full] = ~np.uint64(0)
    if rem:
        mask[full] = (np.uint64(1) << _U64(rem)) - _U64(1)
    return mask


def dense(m: int, n: int, seed: int, stride: int | None = None) -> np.ndarray:
    """m x n matrix with iid Bernoulli(1/2) entries, packed (m, stride) uint64."""
    stride = default_stride(n) if stride is None else stride
    out = np.zeros((m, stride), dtype=np.uint64)
    W = words_per_row(n)
    if m == 0 or W == 0:
        return out
    rows = np.arange(m, dtype=np.uint64)[:, None]
    cols = np.arange(W, dtype=np.uint64)[None, :]
    ctr = (rows << _U64(32)) | cols
    out[:, :W] = mix(_U64(seed) ^ mix(ctr))
    out &= _pad_mask(n, stride)[None, :]
    return out


def bernoulli(m: int, n: int, p: float, seed: int, stride: int | None = None,
              start_col: np.ndarray | None = None, row_block: int = 256) -> np.ndarray:
    """m x n matrix with iid Bernoulli(p) bits, packed (m, stride) uint64.

    ``start_col`` (length m, optional) zeroes row i before column start_col[i].
    """
    stride = default_stride(n) if stride is None else stride
    out = np.zeros((m, stride), dtype=np.uint64)
    if m == 0 or n == 0:
        return out
    thresh = _U64(int(p * float(1 << 53)))
    cols = np.arange(n, dtype=np.uint64)[None, :]
    W = words_per_row(n)
    shifts = (np.arange(64, dtype=np.uint64))
    for r0 in range(0, m, row_block):
        r1 = min(m, r0 + row_block)
        rows = np.arange(r0, r1, dtype=np.uint64)[:, None]
        h = mix(_U64(seed) ^ TAG_P ^ mix((rows << _U64(32)) | cols))
        bits = (h >> _U64(11)) < thresh
        if start_col is not None:
            sc = np.asarray(start_col[r0:r1], dtype=np.int64)[:, None]
            bits &= np.arange(n, dtype=np.int64)[None, :] >= sc
        padded = np.zeros((r1 - r0, W * 64), dtype=np.uint64)
        padded[:, :n] = bits
        padded = padded.reshape(r1 - r0, W, 64)
        out[r0:r1, :W] = np.bitwise_or.reduce(padded << shifts[None, None, :], axis=2)
    return out


def echelon_start(m: int, n: int, frac: float = 0.5) -> np.ndarray:
    """First allowed column of each row of the staircase recipe."""
    i = np.arange(m, dtype=np.float64)
    return np.floor(frac * i * n / max(m, 1)).astype(np.int64)


def echelon(m: int, n: int, p: float, seed: int, frac: float = 0.5,
            stride: int | None = None) -> np.ndarray:
    """Row i zero before column floor(frac*i*n/m), Bernoulli(p) after it."""
    return bernoulli(m, n, p, seed, stride, start_col=echelon_start(m, n, frac))


def derive_seed(seed: int, k: int) -> int:
    """Independent child seed number k of ``seed`` (for B, C factors, batches)."""
    return int(mix(_U64(seed) ^ mix(_U64(k))))


# ---- conversions used by tests (pure data movement, no arithmetic) ----------

def unpack(A: np.ndarray, m: int, n: int) -> np.ndarray:
    """Packed (m, stride) uint64 -> (m, n) uint8 array of 0/1."""
    if m == 0 or n == 0:
        return np.zeros((m, n), dtype=np.uint8)
    W = words_per_row(n)
    b = (A[:m, :W, None] >> np.arange(64, dtype=np.uint64)[None, None, :]) & _U64(1)
    return b.reshape(m, W * 64)[:, :n].astype(np.uint8)


def pack(B: np.ndarray, stride: int | None = None) -> np.ndarray:
    """(m, n) 0/1 array -> packed (m, stride) uint64."""
    B = np.asarray(B, dtype=np.uint64)
    m, n = B.shape
    stride = default_stride(n) if stride is None else stride
    W = words_per_row(n)
    out = np.zeros((m, stride), dtype=np.uint64)
    if m == 0 or n == 0:
        return out
    padded = np.zeros((m, W * 64), dtype=np.uint64)
    padded[:, :n] = B & _U64(1)
    padded = padded.reshape(m, W, 64)
    out[:, :W] = np.bitwise_or.reduce(padded << np.arange(64, dtype=np.uint64)[None, None, :], axis=2)
    return out


def _unit(seed: int, k: int) -> float:
    """Uniform double in [0, 1) from counter k of ``seed`` (top 53 bits)."""
    return float(int(mix(_U64(seed) ^ mix(_U64(k)))) >> 11) * (1.0 / 9007199254740992.0)


def batch_recipe(count: int, base_seed: int):
    """Shapes and densities of a batch of independent matrices (the many-matrix
    workload): rows = floor(exp(U[ln 256, ln 8192])), cols = max(64, 64 *
    round(rows * U[0.5, 2] / 64)), density drawn from {0.5, 0.1, 0.01}, seed of
    matrix i = mix(base_seed + i). Returns a list of (m, n, p, seed)."""
    out = []
    lo, hi = np.log(256.0), np.log(8192.0)
    for i in range(count):
        s = int(mix(_U64((base_seed + i) & 0xFFFFFFFFFFFFFFFF)))
        m = int(np.floor(np.exp(lo + (hi - lo) * _unit(s, 1))))
        n = max(64, 64 * int(round(m * (0.5 + 1.5 * _unit(s, 2)) / 64)))
        p = (0.5, 0.1, 0.01)[min(2, int(3 * _unit(s, 3)))]
        out.append((m, n, p, s))
    return out


def request_recipe(count: int, base_seed: int):
    """Shapes of a stream of requests (the request-stream workload): m =
    floor(exp(U[ln 512, ln 32768])), n = 64 * ceil(m * U[1, 2] / 64), row i zero
    before column floor(0.5 i n / m) and Bernoulli(0.3) after it; seed of request
    i = mix(base_seed + i). Returns a list of (m, n, seed)."""
    out = []
    lo, hi = np.log(512.0), np.log(32768.0)
    for i in range(count):
        s = int(mix(_U64((base_seed + 0x5E5E0000 + i) & 0xFFFFFFFFFFFFFFFF)))
        m = int(np.floor(np.exp(lo + (hi - lo) * _unit(s, 1))))
        n = 64 * int(np.ceil(m * (1.0 + _unit(s, 2)) / 64))
        out.append((m, n, s))
    return out


def arrival_times(count: int, rate: float, seed: int) -> np.ndarray:
    """Poisson arrivals at `rate` per second: cumulative exponential gaps (s)."""
    u = np.array([_unit(seed, 1000 + i) for i in range(count)])
    return np.cumsum(-np.log1p(-u) / rate)
