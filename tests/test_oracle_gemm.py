"""Pins for the oracle's modular product C <- C op A*B mod p (CPU only).

Pinned against: a hand-computed worked example (tests/golden), brute force with
Python integers on tiny inputs, closed forms (rank-1 products, all-ones
matrices, the (p-1)^2 == 1 overflow case), algebraic identities (identity,
associativity, distributivity), the paper's own field GF(2) (nilpotent
matrices), and a Freivalds check that must catch a planted error.
"""
import numpy as np
import pytest

from conftest import load_keyed

import fm_inputs

PRIMES = [2, 3, 7, 251, 65521, 2147483647]


def brute(C, A, B, p, op):
    M, K = len(A), len(A[0]) if len(A) else 0
    N = len(B[0]) if len(B) else 0
    out = []
    for i in range(M):
        row = []
        for j in range(N):
            s = 0
            for l in range(K):
                s += int(A[i][l]) * int(B[l][j])
            c = 0 if C is None else int(C[i][j])
            row.append([s, c + s, c - s][op] % p)
        out.append(row)
    return out


def test_golden_gf7(orc):
    g = load_keyed("gemm_gf7_2x2.txt")
    p = g["p"][0]
    A = np.array(g["A"], dtype=np.uint32).reshape(2, 2)
    B = np.array(g["B"], dtype=np.uint32).reshape(2, 2)
    C = np.array(g["C"], dtype=np.uint32).reshape(2, 2)
    for name, op in (("SET", 0), ("ADD", 1), ("SUB", 2)):
        out = orc.gemm_modp(C, A, B, p, op)
        assert out.ravel().tolist() == g[name], name


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("op", [0, 1, 2])
def test_brute_force_tiny(orc, p, op):
    for seed in range(6):
        dims = fm_inputs.integers(seed, 3, 1, 8, stream=op)
        M, N, K = (int(x) for x in dims)
        A = fm_inputs.uniform_residues(seed, (M, K), p, 1)
        B = fm_inputs.uniform_residues(seed, (K, N), p, 2)
        C = fm_inputs.uniform_residues(seed, (M, N), p, 3)
        out = orc.gemm_modp(C, A, B, p, op)
        assert out.tolist() == brute(C.tolist(), A.tolist(), B.tolist(), p, op)


def test_empty_dimensions(orc):
    p = 65521
    A = np.zeros((3, 0), dtype=np.uint32)
    B = np.zeros((0, 4), dtype=np.uint32)
    C = fm_inputs.uniform_residues(1, (3, 4), p)
    assert np.array_equal(orc.gemm_modp(C, A, B, p, 2), C)
    assert np.array_equal(orc.gemm_modp(C, A, B, p, 0), np.zeros((3, 4), np.uint32))


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_identity(orc, p):
    A = fm_inputs.uniform_residues(2, (13, 13), p)
    I = np.eye(13, dtype=np.uint32)
    assert np.array_equal(orc.gemm_modp(None, I, A, p, 0), A)
    assert np.array_equal(orc.gemm_modp(None, A, I, p, 0), A)
    assert np.array_equal(orc.gemm_modp(A, I, A, p, 2), np.zeros_like(A))


@pytest.mark.parametrize("p", [7, 65521, 2147483647])
def test_rank1_closed_form(orc, p):
    # (u v^T)(w x^T) = (v . w) u x^T: a transposed or swapped operand breaks it
    u = fm_inputs.uniform_residues(1, 5, p, 1).astype(object)
    v = fm_inputs.uniform_residues(1, 6, p, 2).astype(object)
    w = fm_inputs.uniform_residues(1, 6, p, 3).astype(object)
    x = fm_inputs.uniform_residues(1, 4, p, 4).astype(object)
    A = (np.outer(u, v) % p).astype(np.uint32)
    B = (np.outer(w, x) % p).astype(np.uint32)
    vw = int(sum(int(a) * int(b) for a, b in zip(v, w)) % p)
    expect = (np.outer(u, x) * vw % p).astype(np.uint32)
    assert np.array_equal(orc.gemm_modp(None, A, B, p, 0), expect)


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_associativity_distributivity(orc, p):
    A = fm_inputs.uniform_residues(4, (11, 17), p, 1)
    B = fm_inputs.uniform_residues(4, (17, 9), p, 2)
    C = fm_inputs.uniform_residues(4, (9, 6), p, 3)
    D = fm_inputs.uniform_residues(4, (17, 9), p, 4)
    AB_C = orc.gemm_modp(None, orc.gemm_modp(None, A, B, p, 0), C, p, 0)
    A_BC = orc.gemm_modp(None, A, orc.gemm_modp(None, B, C, p, 0), p, 0)
    assert np.array_equal(AB_C, A_BC)
    BD = ((B.astype(np.int64) + D) % p).astype(np.uint32)
    lhs = orc.gemm_modp(None, A, BD, p, 0)
    rhs = orc.gemm_modp(orc.gemm_modp(None, A, B, p, 0), A, D, p, 1)
    assert np.array_equal(lhs, rhs)


@pytest.mark.parametrize("p,K", [(7, 100), (65521, 70000), (2147483647, 1000)])
def test_all_ones_and_overflow(orc, p, K):
    # J_{MxK} J_{KxN} = K J mod p (K > p exercises the reduction)
    J1 = np.ones((3, K), dtype=np.uint32)
    J2 = np.ones((K, 2), dtype=np.uint32)
    assert np.all(orc.gemm_modp(None, J1, J2, p, 0) == K % p)
    # (p-1)^2 == 1 mod p, so K copies of (p-1)*(p-1) sum to K mod p; with
    # p = 2^31-1 and K = 1000 the raw sum exceeds 2^64.
    P1 = np.full((2, K), p - 1, dtype=np.uint32)
    P2 = np.full((K, 3), p - 1, dtype=np.uint32)
    assert np.all(orc.gemm_modp(None, P1, P2, p, 0) == K % p)
    # subtract form: 0 - K mod p
    assert np.all(orc.gemm_modp(np.zeros((2, 3), np.uint32), P1, P2, p, 2) == (-K) % p)


def test_gf2_nilpotent(orc):
    # The paper's own field (Sec. 2.2, "Performance Analysis": GF(2)). For the
    # strictly upper-triangular all-ones N of order n, N^(n-1) has a single one
    # at (0, n-1) and N^n = 0.
    n = 6
    N = np.triu(np.ones((n, n), dtype=np.uint32), 1)
    P = N.copy()
    for _ in range(n - 2):
        P = orc.gemm_modp(None, P, N, 2, 0)
    expect = np.zeros((n, n), dtype=np.uint32)
    expect[0, n - 1] = 1
    assert np.array_equal(P, expect)
    assert not orc.gemm_modp(None, P, N, 2, 0).any()


def test_sub_then_add_inverts(orc):
    p = 65521
    A = fm_inputs.uniform_residues(8, (20, 30), p, 1)
    B = fm_inputs.uniform_residues(8, (30, 25), p, 2)
    C = fm_inputs.uniform_residues(8, (20, 25), p, 3)
    assert np.array_equal(orc.gemm_modp(orc.gemm_modp(C, A, B, p, 2), A, B, p, 1), C)


def test_entries_and_freivalds(orc):
    p = 65521
    A = fm_inputs.uniform_residues(9, (40, 33), p, 1)
    B = fm_inputs.uniform_residues(9, (33, 27), p, 2)
    C = fm_inputs.uniform_residues(9, (40, 27), p, 3)
    full = orc.gemm_modp(C, A, B, p, 2)
    ij = np.array([[0, 0], [39, 26], [17, 5], [3, 20]])
    assert np.array_equal(orc.gemm_modp_entries(C, A, B, p, 2, ij), full[ij[:, 0], ij[:, 1]])
    assert orc.freivalds(full, C, A, B, p, 2)
    bad = full.copy()
    bad[7, 11] = (bad[7, 11] + 1) % p
    assert not orc.freivalds(bad, C, A, B, p, 2)
