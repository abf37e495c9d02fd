"""Pins for the oracle's bit-packed GF(2) matrices and the GF(2) product (CPU only).

The bit-packed layout is the Morton-hybrid order with T' = 32 (Sec. 1; the
experiments of Sec. 2.2 use T' = 32 over the binary field) read 32 entries per
word; the product over GF(2) is gemm_modp with p = 2."""
import os

import numpy as np
import pytest

import fm_inputs
from conftest import ROOT


def _golden():
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", "gf2_pack_entries.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append(tuple(int(x) for x in line.split()))
    return rows


def test_single_entries_land_where_derived_by_hand():
    import oracle
    for lg, i, j, word, bit in _golden():
        n = 32 << lg
        x = np.zeros((n, n), dtype=np.uint32)
        x[i, j] = 1
        w = oracle.gf2_pack(x, lg)
        assert w.size == n * n // 32
        assert np.flatnonzero(w).tolist() == [word]
        assert int(w[word]) == 1 << bit


@pytest.mark.parametrize("rows,cols,lg", [(64, 64, 1), (70, 33, 2), (1, 1, 0), (128, 100, 2)])
def test_pack_round_trip_and_padding(rows, cols, lg):
    import oracle
    x = fm_inputs.uniform_residues(rows * 7 + cols, (rows, cols), 2)
    w = oracle.gf2_pack(x, lg)
    assert np.array_equal(oracle.gf2_unpack(w, lg, rows, cols), x)
    n = 32 << lg
    full = oracle.gf2_unpack(w, lg, n, n)
    assert not full[rows:, :].any() and not full[:, cols:].any()
    # only bit 0 of each entry counts
    assert np.array_equal(oracle.gf2_pack(x + 2 * fm_inputs.uniform_residues(5, (rows, cols), 1000), lg), w)


def test_tile_is_32_consecutive_words_of_row_bits():
    import oracle
    # a full row of ones inside tile (0, 1) of a 64 x 64 matrix: word 32 + u is all ones
    x = np.zeros((64, 64), dtype=np.uint32)
    x[7, 32:] = 1
    w = oracle.gf2_pack(x, 1)
    assert np.flatnonzero(w).tolist() == [32 + 7] and int(w[39]) == 0xFFFFFFFF


@pytest.mark.parametrize("M,N,K", [(5, 7, 9), (33, 40, 65), (64, 1, 130)])
def test_gf2_product_against_bitset_parity(orc, M, N, K):
    # brute force with Python integers as bit sets: C(i, j) = parity of
    # popcount(row i of A AND column j of B), C <- C + A B over GF(2)
    A = fm_inputs.uniform_residues(M + K, (M, K), 2, 1)
    B = fm_inputs.uniform_residues(N + K, (K, N), 2, 2)
    C = fm_inputs.uniform_residues(M + N, (M, N), 2, 3)
    rows = [int("".join(str(int(b)) for b in A[i][::-1]), 2) for i in range(M)]
    cols = [int("".join(str(int(b)) for b in B[:, j][::-1]), 2) for j in range(N)]
    want = np.array([[(int(C[i, j]) + bin(rows[i] & cols[j]).count("1")) & 1 for j in range(N)]
                     for i in range(M)], dtype=np.uint32)
    assert np.array_equal(orc.gemm_modp(C, A, B, 2, 1), want)
    assert np.array_equal(orc.gemm_modp(C, A, B, 2, 2), want)   # -1 = +1 in GF(2)
