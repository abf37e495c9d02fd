"""Pins of the Hilbert-hybrid oracle (the curve variant Sec. 1 compares with the
Morton-hybrid order) against properties that define the Hilbert curve, not
against the oracle's own construction."""
import numpy as np
import pytest

from oracle import hilbert


@pytest.mark.parametrize("m", range(0, 7))
def test_curve_visits_every_cell_once_and_moves_to_a_neighbour(m):
    cells = hilbert.curve(m)
    side = 1 << m
    assert sorted(cells) == [(i, j) for i in range(side) for j in range(side)]
    # a Hilbert curve never jumps: consecutive cells share an edge
    for (i0, j0), (i1, j1) in zip(cells, cells[1:]):
        assert abs(i0 - i1) + abs(j0 - j1) == 1


def test_order_one_and_two_patterns():
    # order 1: the "U" through (0,0), (0,1), (1,1), (1,0); order 2 by hand from
    # that pattern (first quadrant transposed, last reflected on the anti-diagonal)
    assert hilbert.curve(1) == ((0, 0), (0, 1), (1, 1), (1, 0))
    H2 = np.array([[0, 3, 4, 5],
                   [1, 2, 7, 6],
                   [14, 13, 8, 9],
                   [15, 12, 11, 10]])
    assert np.array_equal(hilbert.index_map(2), H2)


@pytest.mark.parametrize("m", range(1, 7))
def test_quadrants_hold_the_smaller_curve(m):
    # the curve enters at (0, 0), leaves at the last row's first cell, and each
    # quadrant holds a quarter of the positions in one contiguous run
    H = hilbert.index_map(m)
    s = 1 << (m - 1)
    q = s * s
    assert H[0, 0] == 0 and H[2 * s - 1, 0] == 4 * q - 1
    for k, (qi, qj) in enumerate(((0, 0), (0, 1), (1, 1), (1, 0))):
        block = H[qi * s:(qi + 1) * s, qj * s:(qj + 1) * s]
        assert block.min() == k * q and block.max() == (k + 1) * q - 1
    # quadrants (0, 1) and (1, 1) hold the order-(m-1) curve as it is
    Hm = hilbert.index_map(m - 1)
    assert np.array_equal(H[0:s, s:2 * s], Hm + q)
    assert np.array_equal(H[s:2 * s, s:2 * s], Hm + 2 * q)
    assert np.array_equal(H[0:s, 0:s], Hm.T)


@pytest.mark.parametrize("rows,cols,m,T", [(7, 5, 2, 2), (16, 16, 2, 4), (30, 17, 3, 4), (1, 1, 0, 1)])
def test_layout_round_trip_and_tile_placement(rows, cols, m, T):
    x = np.arange(1, rows * cols + 1, dtype=np.uint32).reshape(rows, cols)
    flat = hilbert.to_hilbert(x, m, T)
    assert np.array_equal(hilbert.from_hilbert(flat, m, T, rows, cols), x)
    # every tile is one contiguous row-major block at H(I, J) T'^2
    H = hilbert.index_map(m)
    n = (1 << m) * T
    full = np.zeros((n, n), dtype=np.uint32)
    full[:rows, :cols] = x
    for (i, j) in ((0, 0), (rows - 1, cols - 1), (rows // 2, cols // 3)):
        z = int(H[i // T, j // T]) * T * T + (i % T) * T + (j % T)
        assert flat[z] == full[i, j]
