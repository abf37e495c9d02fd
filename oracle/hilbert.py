"""Hilbert-hybrid layout, by the curve's recursive definition (test infrastructure).

Sec. 1 names the Hilbert order as an alternative to the Morton-hybrid order
and picks the latter for its cheaper index conversion. The paper does not
print the curve; this module builds it from the textbook recursion: the
order-0 curve is the single cell (0, 0); the order-k curve of a 2^k x 2^k grid
runs through the quadrants (I, J) = (0, 0), (0, 1), (1, 1), (1, 0) (in units of
s = 2^(k-1) cells), the first holding the order-(k-1) curve transposed, the two
middle ones holding it as it is, the last holding it reflected across the
anti-diagonal. The list of visited cells is built explicitly, so the index of
a cell is its position in that list (no bit manipulation).

A Hilbert-hybrid matrix of side 2^m T' stores tile (I, J) (T' x T' entries,
row-major inside) at H(I, J) * T'^2, with H the order-m curve's index.
"""

from __future__ import annotations

import functools

import numpy as np


@functools.lru_cache(maxsize=None)
def curve(m: int) -> tuple:
    """Cells (I, J) of the order-m curve, in the order the curve visits them."""
    if m == 0:
        return ((0, 0),)
    prev = curve(m - 1)
    s = 1 << (m - 1)
    first = tuple((j, i) for (i, j) in prev)                         # transposed
    second = tuple((i, j + s) for (i, j) in prev)                    # as it is, quadrant (0, 1)
    third = tuple((i + s, j + s) for (i, j) in prev)                 # as it is, quadrant (1, 1)
    fourth = tuple((s - 1 - j + s, s - 1 - i) for (i, j) in prev)    # anti-transposed, quadrant (1, 0)
    return first + second + third + fourth


def index_map(m: int) -> np.ndarray:
    """H as a 2^m x 2^m array: H[I, J] = position of cell (I, J) along the curve."""
    side = 1 << m
    H = np.full((side, side), -1, dtype=np.int64)
    for d, (i, j) in enumerate(curve(m)):
        H[i, j] = d
    return H


def to_hilbert(src: np.ndarray, m: int, T: int) -> np.ndarray:
    """Row-major 2-D array -> flat Hilbert-hybrid array of (2^m T')^2, zero padded."""
    src = np.asarray(src, dtype=np.uint32)
    rows, cols = src.shape
    n = (1 << m) * T
    if rows > n or cols > n:
        raise ValueError("matrix does not fit the grid")
    full = np.zeros((n, n), dtype=np.uint32)
    full[:rows, :cols] = src
    H = index_map(m)
    out = np.empty(n * n, dtype=np.uint32)
    for I in range(1 << m):
        for J in range(1 << m):
            base = int(H[I, J]) * T * T
            out[base:base + T * T] = full[I * T:(I + 1) * T, J * T:(J + 1) * T].reshape(-1)
    return out


def from_hilbert(flat: np.ndarray, m: int, T: int, rows: int, cols: int) -> np.ndarray:
    """Flat Hilbert-hybrid array -> row-major rows x cols corner."""
    flat = np.asarray(flat, dtype=np.uint32)
    n = (1 << m) * T
    if flat.size != n * n:
        raise ValueError("array has the wrong size")
    H = index_map(m)
    full = np.empty((n, n), dtype=np.uint32)
    for I in range(1 << m):
        for J in range(1 << m):
            base = int(H[I, J]) * T * T
            full[I * T:(I + 1) * T, J * T:(J + 1) * T] = flat[base:base + T * T].reshape(T, T)
    return full[:rows, :cols].copy()
