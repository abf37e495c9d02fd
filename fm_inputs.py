"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module only draws random numbers. It holds none of the arithmetic of the
method (no Morton indexing, no modular products, no limb splitting), so both the
CUDA path and the CPU oracle can take their inputs from it without sharing any
computation.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style: draw i of a stream is the
SplitMix64 output function applied to ``base + (i + 1) * golden`` where ``base``
identifies (seed, stream, attempt). Uniform residues in [0, p) are obtained by
rejection: a 64-bit draw ``v`` is kept when ``v < floor(2^64 / p) * p`` and then
mapped to ``v mod p``; a rejected index is redrawn from the next attempt stream.

Workload shapes follow the paper's experiments and the library's target
workloads: i.i.d. uniform residues modulo a prime, random row and column
permutations, random sub-matrix rectangles inside Morton-hybrid matrices
(the paper's experiment draws random start indices and dimensions, Sec. 2.2,
"Performance Analysis"), and batches of GEMM shapes uniform in a range.
"""

from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _mix1(x: int) -> int:
    return int(_mix(np.array([x & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0])


def _base(seed: int, stream: int, attempt: int) -> np.uint64:
    b = _mix1((seed * 0x632BE59BD9B4E019 + 0x1234567) & 0xFFFFFFFFFFFFFFFF)
    b = _mix1(b ^ ((stream + 1) * 0xD1342543DE82EF95))
    b = _mix1(b ^ ((attempt + 1) * 0xA0761D6478BD642F))
    return np.uint64(b)


def raw_u64(seed: int, n: int, stream: int = 0, attempt: int = 0,
            start: int = 0) -> np.ndarray:
    """Draws ``start .. start+n-1`` of the (seed, stream, attempt) sequence."""
    base = _base(seed, stream, attempt)
    idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(base + idx * _GOLDEN)


def uniform_residues(seed: int, shape, p: int, stream: int = 0) -> np.ndarray:
    """i.i.d. uniform residues in [0, p) as uint32, exactly uniform by rejection."""
    if not (2 <= p < (1 << 32)):
        raise ValueError("p must be in [2, 2^32)")
    shape = tuple(int(s) for s in np.atleast_1d(shape)) if not isinstance(shape, int) else (int(shape),)
    n = int(np.prod(shape, dtype=np.int64)) if len(shape) else 1
    out = np.empty(n, dtype=np.uint32)
    pp = np.uint64(p)
    lim_int = ((1 << 64) // p) * p          # == 2^64 when p is a power of two
    lim = np.uint64(lim_int) if lim_int < (1 << 64) else None
    for s in range(0, n, _CHUNK):
        m = min(_CHUNK, n - s)
        v = raw_u64(seed, m, stream, 0, s)
        bad = np.nonzero(v >= lim)[0] if lim is not None else np.zeros(0, np.int64)
        attempt = 1
        while bad.size:
            # redraw only the rejected indices, from the next attempt stream
            redraw = np.array([raw_u64(seed, 1, stream, attempt, s + int(b))[0] for b in bad],
                              dtype=np.uint64)
            v[bad] = redraw
            bad = bad[redraw >= lim]
            attempt += 1
        out[s:s + m] = (v % pp).astype(np.uint32)
    return out.reshape(shape)


def permutation(seed: int, n: int, stream: int = 0) -> np.ndarray:
    """A uniformly random permutation of range(n) as int32 (argsort of random keys)."""
    keys = raw_u64(seed, n, stream)
    return np.argsort(keys, kind="stable").astype(np.int32)


def integers(seed: int, n: int, lo: int, hi: int, stream: int = 0) -> np.ndarray:
    """n integers uniform in [lo, hi] (inclusive), as int64, by rejection."""
    span = hi - lo + 1
    if span <= 0:
        raise ValueError("empty range")
    r = uniform_residues(seed, n, span, stream) if span < (1 << 32) else None
    if r is None:
        raise ValueError("range too large")
    return r.astype(np.int64) + lo


def batch_shapes(seed: int, count: int, lo: int = 32, hi: int = 512,
                 stream: int = 0) -> np.ndarray:
    """``count`` GEMM shapes (M, N, K), each uniform in [lo, hi], as int64 (count, 3)."""
    return integers(seed, 3 * count, lo, hi, stream).reshape(count, 3)


def sub_rectangles(seed: int, count: int, n: int, min_dim: int = 1,
                   stream: int = 0) -> np.ndarray:
    """Random sub-matrix products inside n x n matrices, as rows
    (M, N, K, row0_C, col0_C, row0_A, col0_A, row0_B, col0_B), int64.

    The three extents are uniform in [min_dim, n]; each start is uniform among
    the positions that keep the rectangle inside the matrix.
    """
    dims = integers(seed, 3 * count, min_dim, n, stream).reshape(count, 3)
    u = raw_u64(seed, 6 * count, stream + 1).reshape(count, 6)
    out = np.zeros((count, 9), dtype=np.int64)
    for t in range(count):
        M, N, K = (int(x) for x in dims[t])
        out[t, 0:3] = (M, N, K)
        spans = (n - M + 1, n - N + 1, n - M + 1, n - K + 1, n - K + 1, n - N + 1)
        for q in range(6):
            out[t, 3 + q] = int(u[t, q]) % spans[q]
    return out


def batch_workload(seed: int, count: int = 4096, lo: int = 32, hi: int = 512,
                   big: int = 16384) -> tuple:
    """The independent-call batch: ``count`` products with M, N, K uniform in
    [lo, hi]. Call c writes the top-left M x N corner of its own hi x hi cell of
    a C matrix with ``cells`` x ``cells`` cells (cells the smallest power of two
    with cells^2 >= count; cell c at row (c // cells) * hi, column
    (c % cells) * hi); its A and B parts are random rectangles of two shared
    big x big matrices (reads may overlap).

    Returns (rows, cells): rows as int64 (count, 9) =
    (M, N, K, row0_C, col0_C, row0_A, col0_A, row0_B, col0_B)."""
    cells = 1
    while cells * cells < count:
        cells *= 2
    shapes = batch_shapes(seed, count, lo, hi)
    offs = raw_u64(seed, 4 * count, 9).reshape(count, 4)
    out = np.zeros((count, 9), dtype=np.int64)
    for c in range(count):
        M, N, K = (int(x) for x in shapes[c])
        out[c] = (M, N, K, (c // cells) * hi, (c % cells) * hi,
                  int(offs[c, 0]) % (big - M + 1), int(offs[c, 1]) % (big - K + 1),
                  int(offs[c, 2]) % (big - K + 1), int(offs[c, 3]) % (big - N + 1))
    return out, cells
