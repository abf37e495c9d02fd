"""Pins for the oracle's Morton-hybrid index and layout conversion (CPU only).

Pinned against: hand-derived tables (tests/golden), the paper's Step-1 quadrant
offsets and in-tile offset, exhaustive bijection, and the sigma = 112 reading.
"""
import numpy as np
import pytest

from conftest import load_table

import fm_inputs


@pytest.mark.parametrize("name,m,T", [("morton_4x4_T1.txt", 2, 1),
                                      ("morton_8x8_T4.txt", 1, 4),
                                      ("morton_8x8_T2.txt", 2, 2)])
def test_golden_tables(orc, name, m, T):
    table = load_table(name)
    n = (1 << m) * T
    assert len(table) == n
    for i in range(n):
        for j in range(n):
            assert orc.encode(i, j, m, T) == table[i][j], (i, j)
            assert orc.extract_i(table[i][j], m, T) == i
            assert orc.extract_j(table[i][j], m, T) == j


def test_sigma_112_reading(orc):
    # Sec. 2.1 (P2) names a contained base-case block starting at sigma = 112 in
    # a T' = 4 example whose figure is not available. By the layout, 112 / 16 = 7
    # is tile Z(1, 3) of a 4 x 4 tile grid, i.e. Cartesian (4, 12) of a 16 x 16.
    assert orc.encode(4, 12, 2, 4) == 112
    assert (orc.extract_i(112, 2, 4), orc.extract_j(112, 2, 4)) == (4, 12)


@pytest.mark.parametrize("T,mmax", [(1, 6), (2, 6), (4, 6), (3, 4), (32, 3)])
def test_bijection_exhaustive(orc, T, mmax):
    for m in range(0, mmax + 1):
        n = (1 << m) * T
        ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        z = orc.encode_many(ii.ravel(), jj.ravel(), m, T)
        assert np.array_equal(np.sort(z), np.arange(n * n, dtype=np.uint64))
        bi, bj = orc.extract_many(z, m, T)
        assert np.array_equal(bi, ii.ravel()) and np.array_equal(bj, jj.ravel())


@pytest.mark.parametrize("T,m", [(1, 4), (2, 3), (4, 3)])
def test_step1_quadrant_offsets(orc, T, m):
    # Sec. 2.2 Step 1: quadrant q of an aligned block (alpha, lambda) starts at
    # alpha + q * lambda / 4, in the order NW, NE, SW, SE; every aligned block is
    # a contiguous index range.
    n = (1 << m) * T
    size = n
    while size > T:
        h = size // 2
        for bi in range(0, n, size):
            for bj in range(0, n, size):
                alpha = orc.encode(bi, bj, m, T)
                lam = size * size
                starts = [orc.encode(bi, bj, m, T), orc.encode(bi, bj + h, m, T),
                          orc.encode(bi + h, bj, m, T), orc.encode(bi + h, bj + h, m, T)]
                assert starts == [alpha + q * lam // 4 for q in range(4)]
                zs = [orc.encode(bi + a, bj + b, m, T) for a in range(size) for b in range(size)]
                assert sorted(zs) == list(range(alpha, alpha + lam))
        size = h


@pytest.mark.parametrize("T,m", [(4, 2), (8, 2), (3, 2)])
def test_in_tile_row_major(orc, T, m):
    # Sec. 2.1 P2: in a T' x T' block starting at sigma, (i, j) is sigma + i*T' + j;
    # Cor. 2.3: an aligned T' x T' sub-matrix is row-major.
    n = (1 << m) * T
    for I in range(0, n, T):
        for J in range(0, n, T):
            sigma = orc.encode(I, J, m, T)
            assert sigma % (T * T) == 0
            for i in range(T):
                for j in range(T):
                    assert orc.encode(I + i, J + j, m, T) == sigma + i * T + j


def test_to_from_morton_roundtrip_and_padding(orc):
    rng_src = fm_inputs.uniform_residues(3, (37, 53), 65521)
    m, T = 2, 16
    z = orc.to_morton(rng_src, m, T)
    back = orc.from_morton(z, m, T, 37, 53)
    assert np.array_equal(back, rng_src)
    # every padded position holds zero, every real position its value
    n = (1 << m) * T
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    zz = orc.encode_many(ii.ravel(), jj.ravel(), m, T)
    full = np.zeros((n, n), dtype=np.uint32)
    full[:37, :53] = rng_src
    assert np.array_equal(z[zz.astype(np.int64)], full.ravel())


def test_to_morton_golden_permutation(orc):
    table = np.array(load_table("morton_8x8_T4.txt"))
    src = np.arange(64, dtype=np.uint32).reshape(8, 8) * 3 + 1
    z = orc.to_morton(src, 1, 4)
    for i in range(8):
        for j in range(8):
            assert z[table[i, j]] == src[i, j]


def test_permute_matches_permutation_matrices(orc):
    # out = P X Q with P[i, rp[i]] = 1 and Q[cp[j], j] = 1, through the product.
    p = 65521
    X = fm_inputs.uniform_residues(5, (9, 7), p)
    rp = fm_inputs.permutation(5, 9, 1)
    cp = fm_inputs.permutation(5, 7, 2)
    P = np.zeros((9, 9), dtype=np.uint32)
    P[np.arange(9), rp] = 1
    Q = np.zeros((7, 7), dtype=np.uint32)
    Q[cp, np.arange(7)] = 1
    PX = orc.gemm_modp(None, P, X, p, orc.OP_SET)
    PXQ = orc.gemm_modp(None, PX, Q, p, orc.OP_SET)
    assert np.array_equal(orc.permute(X, rp, cp), PXQ)
    # composition of gathers
    rp2 = fm_inputs.permutation(6, 9, 1)
    cp2 = fm_inputs.permutation(6, 7, 2)
    assert np.array_equal(orc.permute(orc.permute(X, rp, cp), rp2, cp2),
                          orc.permute(X, rp[rp2], cp[cp2]))
    assert np.array_equal(orc.permute(X, None, None), X)
