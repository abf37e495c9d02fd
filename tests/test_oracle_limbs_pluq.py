"""Pins for the oracle's limb split and rank-revealing PLUQ (CPU only)."""
import numpy as np
import pytest

import fm_inputs


def test_limb_counts_and_bounds():
    from oracle import limbs
    assert [limbs.n_limbs(p) for p in (2, 251, 257, 65521, 65537, 2147483647)] == [1, 1, 2, 2, 3, 4]
    assert limbs.bounds(2) == (-32896, 32639)
    assert limbs.bounds(4) == (-128 * 16843009, 127 * 16843009)


def test_split_exhaustive_65521():
    from oracle import limbs
    p = 65521
    x = np.arange(p, dtype=np.int64)
    d = limbs.split(x, p)
    assert d.shape == (2, p) and d.dtype == np.int8
    r = limbs.recombine(d)
    lo, hi = limbs.bounds(2)
    assert r.min() >= lo and r.max() <= hi
    assert np.array_equal(r % p, x)
    # representative rule: x itself up to Hi, x - p above it
    assert np.array_equal(r[:hi + 1], x[:hi + 1])
    assert np.array_equal(r[hi + 1:], x[hi + 1:] - p)


@pytest.mark.parametrize("p", [257, 4099, 32771, 65521, 65533, 65535])
def test_two_limb_digit_sum_bound(p):
    # every two-limb modulus p < 2^16 keeps d0 + d1 in [-255, 254] (d0 = d1 = -128
    # would need the representative -32896 < 32640 - p), so a Karatsuba middle
    # term (d0 + d1)(e0 + e1) is at most 255^2 = 65025 in magnitude
    from oracle import limbs
    d = limbs.split(np.arange(p, dtype=np.int64), p).astype(np.int64)
    s = d[0] + d[1]
    assert s.min() >= -255 and s.max() <= 254
    if p >= 65280:  # representative -32640 (d0 = -128, d1 = -127) is x = p - 32640
        assert s[p - 32640] == -255
    assert 256 * 255 * 255 + p <= 1 << 24  # a 256-term middle chunk plus the carry is exact


def test_split_31bit_random_and_extremes():
    from oracle import limbs
    p = 2147483647
    _, hi = limbs.bounds(4)
    x = np.concatenate([fm_inputs.uniform_residues(1, 200000, p).astype(np.int64),
                        np.array([0, 1, 127, 128, hi, hi + 1, p - 2, p - 1], dtype=np.int64)])
    d = limbs.split(x, p)
    r = limbs.recombine(d)
    assert np.array_equal(r % p, x)
    assert d.min() >= -128 and d.max() <= 127


@pytest.mark.parametrize("p", [65521, 2147483647, 257])
def test_limb_products_reproduce_modular_product(orc, p):
    # sum_s 256^s sum_{i+j=s} A_i B_j == A_r B_r exactly; mod p it is A*B mod p
    from oracle import limbs
    A = fm_inputs.uniform_residues(2, (9, 31), p, 1)
    B = fm_inputs.uniform_residues(2, (31, 7), p, 2)
    dA, dB = limbs.split(A, p), limbs.split(B, p)
    w = dA.shape[0]
    total = np.zeros((9, 7), dtype=object)
    for i in range(w):
        for j in range(w):
            P = dA[i].astype(np.int64) @ dB[j].astype(np.int64)
            total = total + P.astype(object) * (256 ** (i + j))
    got = np.array([[int(v) % p for v in row] for row in total], dtype=np.uint32)
    assert np.array_equal(got, orc.gemm_modp(None, A, B, p, 0))


def _check_pluq(orc, A, p):
    rp, cp, L, U, r = orc.pluq(A, p)
    assert sorted(rp.tolist()) == list(range(A.shape[0]))
    assert sorted(cp.tolist()) == list(range(A.shape[1]))
    LU = orc.gemm_modp(None, L, U, p, 0)
    assert np.array_equal(orc.permute(A, rp, cp), LU)
    for t in range(r):
        assert L[t, t] == 1 and not L[:t, t].any()
        assert U[t, t] != 0 and not U[t, :t].any()
    return r


def test_pluq_special_cases(orc):
    p = 65521
    assert _check_pluq(orc, np.zeros((5, 7), np.uint32), p) == 0
    assert _check_pluq(orc, np.eye(6, dtype=np.uint32), p) == 6
    u = fm_inputs.uniform_residues(1, 8, p, 1).astype(np.int64)
    v = fm_inputs.uniform_residues(1, 5, p, 2).astype(np.int64)
    u[0] = 1
    v[0] = 1
    assert _check_pluq(orc, (np.outer(u, v) % p).astype(np.uint32), p) == 1
    # cases that need a permutation whatever the pivot rule: with an all-zero
    # first row, U's nonzero first row can only come from row 1 (P is not the
    # identity); with an all-zero first column, U(0, 0) != 0 needs another
    # column first (Q is not the identity)
    A = np.array([[0, 0], [5, 7]], np.uint32)
    assert _check_pluq(orc, A, p) == 1 and orc.pluq(A, p)[0][0] == 1
    A = np.array([[0, 2, 4], [0, 1, 9]], np.uint32)
    assert _check_pluq(orc, A, p) == 2 and orc.pluq(A, p)[1][0] != 0


@pytest.mark.parametrize("p", [2, 3, 65521])
def test_pluq_rank_deficient_against_library_rank(orc, p):
    sympy = pytest.importorskip("sympy")
    from sympy.polys.matrices import DomainMatrix
    from sympy import GF
    for seed in range(8):
        m, n, r = (int(x) for x in fm_inputs.integers(seed, 3, 1, 9, stream=p % 97))
        r = min(r, m, n)
        X = fm_inputs.uniform_residues(seed, (m, r), p, 1)
        Y = fm_inputs.uniform_residues(seed, (r, n), p, 2)
        A = orc.gemm_modp(None, X, Y, p, 0)
        rank = _check_pluq(orc, A, p)
        dm = DomainMatrix([[GF(p)(int(v)) for v in row] for row in A.tolist()], (m, n), GF(p))
        assert rank == dm.rank()
        assert rank <= r


@pytest.mark.parametrize("p", [65537, 1000003, 16777259, 2147483647, 65534])
def test_pairwise_karatsuba_digit_sums_and_identity(orc, p):
    # Karatsuba over every pair of limbs (the tensor-core residue form for w >= 2,
    # p >= 2^16 or even): a digit sum d_i + d_j stays in [-256, 254], so a term of
    # a pair product is at most 2^16 and a 256-term chunk at most 2^24 (exact in
    # FP32); and sum_i w_ii A_i B_i + sum_{i<j} 256^(i+j) (A_i + A_j)(B_i + B_j)
    # with w_ii = 256^(2i) - sum_{j != i} 256^(i+j) equals the product of the
    # representatives over the integers, hence A*B mod p
    from oracle import limbs
    w = limbs.n_limbs(p)
    _, hi = limbs.bounds(w)
    x = np.concatenate([fm_inputs.uniform_residues(3, 100000, p).astype(np.int64),
                        np.array([0, 1, 127, 128, hi, hi + 1, p - 2, p - 1], dtype=np.int64)])
    x = x[x < p]
    d = limbs.split(x, p).astype(np.int64)
    for i in range(w):
        for j in range(i + 1, w):
            s = d[i] + d[j]
            assert s.min() >= -256 and s.max() <= 254
    assert 256 * 256 * 256 <= 1 << 24
    A = fm_inputs.uniform_residues(4, (7, 40), p, 1)
    B = fm_inputs.uniform_residues(4, (40, 5), p, 2)
    dA, dB = limbs.split(A, p).astype(object), limbs.split(B, p).astype(object)
    total = np.zeros((7, 5), dtype=object)
    for i in range(w):
        wii = 256 ** (2 * i) - sum(256 ** (i + j) for j in range(w) if j != i)
        total = total + wii * (dA[i] @ dB[i])
        for j in range(i + 1, w):
            total = total + 256 ** (i + j) * ((dA[i] + dA[j]) @ (dB[i] + dB[j]))
    rA = limbs.recombine(limbs.split(A, p)).astype(object)
    rB = limbs.recombine(limbs.split(B, p)).astype(object)
    assert np.array_equal(total, rA @ rB)
    got = np.array([[int(v) % p for v in row] for row in total], dtype=np.uint32)
    assert np.array_equal(got, orc.gemm_modp(None, A, B, p, 0))
