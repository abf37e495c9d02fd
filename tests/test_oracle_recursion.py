"""Pins for the oracle's aligned / contained recursion (Sec. 2.2, Steps 1-4).

Pinned against: brute-force exact cover of the (i, j, l) index space, the
paper's propositions (every base-case part lies inside one row-major tile:
Prop. and Cor. of Sec. 2.1; at most 64 combinations per level: Step 3), Step 2
against brute-force rectangle clipping, and a numeric check that running the
base cases with the paper's row-major offset (Sec. 2.1 P2) reproduces the
modular product.
"""
import itertools

import numpy as np
import pytest

import fm_inputs


def _rect_in_one_tile(i0, j0, r, c, T):
    return (i0 // T == (i0 + r - 1) // T) and (j0 // T == (j0 + c - 1) // T)


def _cases(n, count, seed):
    for row in fm_inputs.sub_rectangles(seed, count, n):
        M, N, K, iA, jA, iB, jB, iC, jC = (int(x) for x in row)
        yield (iA, jA, M, N), (iB, jB, M, K), (iC, jC, K, N)


@pytest.mark.parametrize("m,T", [(0, 4), (1, 2), (2, 2), (2, 3), (3, 1), (1, 5)])
def test_exact_cover_and_containment(m, T):
    from oracle import recursion
    n = (1 << m) * T
    for sA, sB, sC in _cases(n, 12, seed=m * 10 + T):
        rec = recursion.Recursion(m, T, sA, sB, sC)
        leaves = rec.run()
        M, N, K = sA[2], sA[3], sB[3]
        seen = np.zeros((M, N, K), dtype=np.int32)
        for lf in leaves:
            seen[lf.i_lo:lf.i_hi, lf.j_lo:lf.j_hi, lf.l_lo:lf.l_hi] += 1
            for P in (lf.A, lf.B, lf.C):
                assert P.r > 0 and P.c > 0
                assert _rect_in_one_tile(P.i0, P.j0, P.r, P.c, T), "scattered base part"
            # the three parts agree with the local ranges
            assert (lf.A.r, lf.A.c) == (lf.i_hi - lf.i_lo, lf.j_hi - lf.j_lo)
            assert (lf.B.r, lf.B.c) == (lf.i_hi - lf.i_lo, lf.l_hi - lf.l_lo)
            assert (lf.C.r, lf.C.c) == (lf.l_hi - lf.l_lo, lf.j_hi - lf.j_lo)
            assert lf.A.i0 == sA[0] + lf.i_lo and lf.A.j0 == sA[1] + lf.j_lo
            assert lf.B.i0 == sB[0] + lf.i_lo and lf.B.j0 == sB[1] + lf.l_lo
            assert lf.C.i0 == sC[0] + lf.l_lo and lf.C.j0 == sC[1] + lf.j_lo
        assert np.all(seen == 1), "every (i, j, l) exactly once"
        assert rec.max_children <= 64


def test_step2_against_clipping(orc):
    from oracle import recursion
    m, T = 3, 2
    n = (1 << m) * T
    for (i0, j0, r, c), _, _ in _cases(n, 40, seed=77):
        sigma = orc.encode(i0, j0, m, T)
        S = recursion.Part(sigma, r, c, i0, j0)
        size = n
        while size > T:
            for bi in range(0, n, size):
                for bj in range(0, n, size):
                    alpha = orc.encode(bi, bj, m, T)
                    # the part of S inside this block, clipped by brute force
                    ci0, ci1 = max(i0, bi), min(i0 + r, bi + size)
                    cj0, cj1 = max(j0, bj), min(j0 + c, bj + size)
                    if ci0 >= ci1 or cj0 >= cj1:
                        continue
                    inner = recursion.Part(orc.encode(ci0, cj0, m, T), ci1 - ci0, cj1 - cj0,
                                           ci0, cj0)
                    parts = recursion.step2_split(alpha, size * size, inner, m, T)
                    h = size // 2
                    quads = [(bi, bj), (bi, bj + h), (bi + h, bj), (bi + h, bj + h)]
                    for P, (qi, qj) in zip(parts, quads):
                        ei0, ei1 = max(ci0, qi), min(ci1, qi + h)
                        ej0, ej1 = max(cj0, qj), min(cj1, qj + h)
                        er, ec = max(ei1 - ei0, 0), max(ej1 - ej0, 0)
                        if er == 0 or ec == 0:
                            assert P.r == 0 or P.c == 0
                        else:
                            assert (P.i0, P.j0, P.r, P.c) == (ei0, ej0, er, ec)
                            assert P.sigma == orc.encode(ei0, ej0, m, T)
            size //= 2


def test_aligned_product_has_no_extra_calls():
    # Aligned sub-matrices: every base case is a full tile product, and there are
    # (M/T')(N/T')(K/T') of them (Table 1's "0 % more calls" case).
    from oracle import recursion
    m, T = 2, 4
    leaves = recursion.leaves(m, T, (4, 0, 8, 12), (0, 4, 8, 4), (8, 0, 4, 12))
    assert len(leaves) == (8 // T) * (12 // T) * (4 // T)
    for lf in leaves:
        assert (lf.i_hi - lf.i_lo, lf.j_hi - lf.j_lo, lf.l_hi - lf.l_lo) == (T, T, T)


@pytest.mark.parametrize("m,T,p", [(2, 2, 65521), (2, 3, 7), (1, 4, 2)])
def test_base_cases_reproduce_the_product(orc, m, T, p):
    # Run every base case as a plain row-major triple loop on the Morton arrays,
    # addressing entry (i, j) of a contained part as sigma + i*T' + j (Sec. 2.1 P2),
    # and compare the accumulated S_A with the definition.
    from oracle import recursion
    n = (1 << m) * T
    for t, (sA, sB, sC) in enumerate(_cases(n, 6, seed=5 + T)):
        A = fm_inputs.uniform_residues(t, (n, n), p, 1)
        B = fm_inputs.uniform_residues(t, (n, n), p, 2)
        C = fm_inputs.uniform_residues(t, (n, n), p, 3)
        zA = orc.to_morton(A, m, T).astype(np.int64)
        zB = orc.to_morton(B, m, T)
        zC = orc.to_morton(C, m, T)
        for lf in recursion.leaves(m, T, sA, sB, sC):
            for i in range(lf.A.r):
                for j in range(lf.A.c):
                    s = 0
                    for l in range(lf.B.c):
                        s += int(zB[lf.B.sigma + i * T + l]) * int(zC[lf.C.sigma + l * T + j])
                    zA[lf.A.sigma + i * T + j] = (zA[lf.A.sigma + i * T + j] + s) % p
        got = orc.from_morton(zA.astype(np.uint32), m, T, n, n)
        iA, jA, M, N = sA
        iB, jB, _, K = sB
        iC, jC, _, _ = sC
        expect = A.copy()
        expect[iA:iA + M, jA:jA + N] = orc.gemm_modp(
            A[iA:iA + M, jA:jA + N], B[iB:iB + M, jB:jB + K], C[iC:iC + K, jC:jC + N], p, 1)
        assert np.array_equal(got, expect)


def test_leaves_equal_interval_partition_cells():
    # The leaves are exactly the cells of three interval partitions: i cut at the
    # tile-row boundaries of A and B, j at the tile-column boundaries of A and C,
    # l at the tile-column boundaries of B and the tile-row boundaries of C.
    from oracle import recursion

    def cuts(length, offs, T):
        pts = {0, length}
        for o in offs:
            pts |= {x - o for x in range(0, o + length + T, T) if 0 < x - o < length}
        pts = sorted(pts)
        return list(zip(pts[:-1], pts[1:]))

    m, T = 3, 2
    n = (1 << m) * T
    for sA, sB, sC in _cases(n, 25, seed=31):
        M, N, K = sA[2], sA[3], sB[3]
        cells = {(a, b, c) for a, b, c in itertools.product(
            cuts(M, (sA[0], sB[0]), T), cuts(N, (sA[1], sC[1]), T), cuts(K, (sB[1], sC[0]), T))}
        got = {((lf.i_lo, lf.i_hi), (lf.j_lo, lf.j_hi), (lf.l_lo, lf.l_hi))
               for lf in recursion.leaves(m, T, sA, sB, sC)}
        assert got == cells


def test_default_calls_aligned_equals_tile_count():
    from oracle import recursion
    assert recursion.default_calls(32, 128, 64, 256) == 4 * 2 * 8
    assert recursion.default_calls(32, 0, 64, 256) == 0
    assert recursion.default_calls(32, 5, 7, 9) == 1
