"""GPU parity of the TU / PLUQ decomposition (fm_pluq) against the oracle.

Parity for a factorisation with many valid outputs (Sec. 1 defers TURBO's exact
outputs; reading R13) is the identity P A Q = L U with L unit lower trapezoidal,
U upper trapezoidal with a nonzero diagonal, and the rank equal to the oracle's.
"""
import numpy as np
import pytest

import fm_inputs
from gpu_util import MortonMatrix, grid_for, lib_and_device, to_dev, to_host

pytestmark = pytest.mark.gpu

P16 = 65521


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def run_pluq(env, A, p, lt):
    fm, dev = env
    m, n = A.shape
    M = MortonMatrix(fm, dev, grid_for(m, n, lt), lt)
    M.load(A)
    rp = to_dev(np.zeros(m, np.int32), dev)
    cp = to_dev(np.zeros(n, np.int32), dev)
    r = fm.fm_pluq(M.m, m, n, p, rp, cp)
    assert fm.fm_get_last_device_status() == 0
    return r, M.read(m, n), to_host(rp).view(np.int32), to_host(cp).view(np.int32)


def check_factors(orc, A, p, r, F, rp, cp):
    m, n = A.shape
    assert sorted(rp.tolist()) == list(range(m))
    assert sorted(cp.tolist()) == list(range(n))
    L = np.tril(F[:, :r], -1).astype(np.uint32)
    L[np.arange(r), np.arange(r)] = 1
    U = np.triu(F[:r, :]).astype(np.uint32)
    assert np.all(np.diag(U[:, :r]) != 0)
    assert np.array_equal(orc.permute(A, rp, cp), orc.gemm_modp(None, L, U, p, 0))


def low_rank(seed, m, n, r, p):
    X = fm_inputs.uniform_residues(seed, (m, r), p, 1)
    Y = fm_inputs.uniform_residues(seed, (r, n), p, 2)
    return X, Y


@pytest.mark.parametrize("m,n,rk,lt", [(300, 200, 150, 6), (200, 300, 200, 6), (256, 256, 256, 7),
                                       (130, 400, 60, 5), (517, 129, 129, 4), (64, 64, 0, 6)])
def test_pluq_small_against_oracle(env, orc, m, n, rk, lt):
    for p in (P16, 3, 2147483647):
        X, Y = low_rank(m + n + rk, m, n, max(rk, 1), p)
        A = orc.gemm_modp(None, X, Y, p, 0) if rk else np.zeros((m, n), np.uint32)
        r, F, rp, cp = run_pluq(env, A, p, lt)
        _, _, _, _, r_oracle = orc.pluq(A, p)
        assert r == r_oracle, (p, r, r_oracle)
        check_factors(orc, A, p, r, F, rp, cp)


def test_pluq_zero_columns_and_rows(env, orc):
    # whole zero columns inside and across panels, zero rows, duplicated rows
    p = P16
    m, n = 260, 300
    A = fm_inputs.uniform_residues(7, (m, n), p)
    A[:, [0, 5, 127, 128, 200, 299]] = 0
    A[[3, 100, 259], :] = 0
    A[50] = A[10]
    r, F, rp, cp = run_pluq(env, A, p, 6)
    _, _, _, _, r_oracle = orc.pluq(A, p)
    assert r == r_oracle
    check_factors(orc, A, p, r, F, rp, cp)


def test_config5_tu_16384x12288_rank_10000(env, orc):
    # TU of a 16384 x 12288 matrix over GF(65521) built as the product of seeded
    # uniform 16384 x 10000 and 10000 x 12288 factors (rank 10000 w.h.p.): the
    # product itself and every trailing update run through fm_gemm_modp.
    import torch
    fm, dev = env
    m, n, k, p = 16384, 12288, 10000, P16
    X, Y = low_rank(5, m, n, k, p)
    lt = 7
    MX = MortonMatrix(fm, dev, grid_for(m, k, lt), lt, fill=X)
    MY = MortonMatrix(fm, dev, grid_for(k, n, lt), lt, fill=Y)
    MA = MortonMatrix(fm, dev, grid_for(m, n, lt), lt)
    fm.fm_gemm_modp(MA.sub(0, 0, m, n), MX.sub(0, 0, m, k), MY.sub(0, 0, k, n), p, 0,
                    fm.FM_ALGO_LIMB_TC)
    A = MA.read(m, n)
    del MX, MY
    # the product is right (sampled entries against the oracle)
    ij = np.stack([fm_inputs.integers(1, 200, 0, m - 1, 1), fm_inputs.integers(1, 200, 0, n - 1, 2)], 1)
    assert np.array_equal(A[ij[:, 0], ij[:, 1]], orc.gemm_modp_entries(None, X, Y, p, 0, ij))
    rp = torch.zeros(m, dtype=torch.int32, device=dev)
    cp = torch.zeros(n, dtype=torch.int32, device=dev)
    r = fm.fm_pluq(MA.m, m, n, p, rp, cp)
    assert fm.fm_get_last_device_status() == 0
    assert r == k
    F = MA.read(m, n)
    rp, cp = to_host(rp).view(np.int32), to_host(cp).view(np.int32)
    assert sorted(rp.tolist()) == list(range(m)) and sorted(cp.tolist()) == list(range(n))
    # Freivalds: (P A Q) x == L (U x) for random x, error probability <= 1/p per trial
    PAQ = orc.permute(A, rp, cp)
    Lfac = np.tril(F[:, :r], -1)
    Lfac[np.arange(r), np.arange(r)] = 1
    Ufac = np.triu(F[:r, :])
    assert np.all(np.diag(Ufac[:, :r]) != 0)
    assert not F[r:, r:].any()
    for t in range(2):
        x = fm_inputs.uniform_residues(9, n, p, 100 + t)
        lhs = orc.matvec_modp(PAQ, x, p)
        rhs = orc.matvec_modp(Lfac.astype(np.uint32), orc.matvec_modp(Ufac.astype(np.uint32), x, p), p)
        assert np.array_equal(lhs, rhs)


def _trace_pluq(env, A, p, lt, tmp_path):
    import os
    log = tmp_path / "pluq_trace.txt"
    os.environ["FM_TRACE"] = str(log)
    try:
        out = run_pluq(env, A, p, lt)
    finally:
        del os.environ["FM_TRACE"]
    line = [x for x in log.read_text().splitlines() if "pluq m=" in x][-1]
    fast = int(line.split("columns: ")[1].split(" diagonal-block")[0])
    searched = int(line.split("diagonal-block, ")[1].split(" searched")[0])
    zero = int(line.split("searched, ")[1].split(" zero")[0])
    return out, fast, searched, zero


@pytest.mark.parametrize("case", ["searched_after_block", "low_rank_after_blocks"])
def test_pluq_look_ahead_stream(env, orc, tmp_path, case):
    # Behind the first outer block (columns 0..511) the look-ahead stream still
    # updates columns 1024.. while the next block's panels factor. Then (a) a zero
    # diagonal pivot at column 650 (row 650 repeats row 5 in the leading 651
    # columns) sends panel 5 to the search, whose row swaps reach every column
    # and must wait for that stream; (b) rank 700: after block 1 ends early the
    # panels past the rank start blocks further right, whose columns the stream
    # may still hold. Both against the oracle's rank and P A Q = L U.
    p, lt, m, n = P16, 6, 1200, 1400
    if case == "searched_after_block":
        A = fm_inputs.uniform_residues(13, (m, n), p)
        A[650, :651] = A[5, :651]
    else:
        X, Y = low_rank(14, m, n, 700, p)
        A = orc.gemm_modp(None, X, Y, p, 0)
    (r, F, rp, cp), fast, searched, zero = _trace_pluq(env, A, p, lt, tmp_path)
    _, _, _, _, r_oracle = orc.pluq(A, p)
    assert r == r_oracle
    check_factors(orc, A, p, r, F, rp, cp)
    if case == "searched_after_block":
        assert searched >= 1 and fast >= 8
    else:
        assert zero >= 4


@pytest.mark.parametrize("case", ["dense", "zero_first_pivot", "zero_mid_pivot", "tiny_field", "low_rank"])
def test_pluq_diagonal_block_and_search_paths(env, orc, tmp_path, case):
    # A full panel whose 128 diagonal pivots are nonzero factors by the
    # diagonal-block path (one-CTA LU of the 128 x 128 block, L21 = A21 U11^-1);
    # a zero pivot on the diagonal -- at its first column, in the middle of the
    # block (row 70 of the leading 71 columns repeats row 3 there), or often in
    # GF(3) -- sends the panel to the column-by-column search; a panel with no
    # nonzero left (rank 200 of 384 columns: the third panel) is skipped. All
    # give a valid P A Q = L U with the oracle's rank.
    p, lt, m, n = P16, 6, 400, 384
    A = fm_inputs.uniform_residues(11, (m, n), p)
    if case == "zero_first_pivot":
        A[0, 0] = 0
    elif case == "zero_mid_pivot":
        A[70, :71] = A[3, :71]
    elif case == "tiny_field":
        p = 3
        A = A % 3
    elif case == "low_rank":  # rank 200: the last panel holds no nonzero once 200 pivots are out
        X, Y = low_rank(12, m, n, 200, p)
        A = orc.gemm_modp(None, X, Y, p, 0)
    (r, F, rp, cp), fast, searched, zero = _trace_pluq(env, A, p, lt, tmp_path)
    _, _, _, _, r_oracle = orc.pluq(A, p)
    assert r == r_oracle
    check_factors(orc, A, p, r, F, rp, cp)
    if case == "dense":
        assert fast == 3 and searched == 0 and zero == 0
    elif case in ("zero_first_pivot", "zero_mid_pivot"):
        assert searched >= 1 and fast >= 1
    elif case == "low_rank":
        assert (fast, searched, zero) == (1, 1, 1)
    else:
        assert searched >= 1


@pytest.mark.parametrize("m,n,rk,lt,p", [(700, 900, 700, 6, P16), (1100, 700, 700, 7, P16), (900, 1300, 450, 6, P16),
                                         (600, 640, 600, 5, 2147483647), (700, 900, 700, 6, 3)])
def test_pluq_outer_blocks(env, orc, m, n, rk, lt, p):
    # Panels grouped in blocks of four (columns behind a block updated once
    # with K = its pivots; inside the block panel by panel): full-rank wide and
    # tall matrices (blocks of four full panels, a last block of fewer),
    # rank 450 (a block that ends early on a panel with 66 pivots), p = 2^31 - 1,
    # and GF(3) (searched panels, blocks ending on short panels)
    X, Y = low_rank(m * 3 + n + rk, m, n, rk, p)
    A = orc.gemm_modp(None, X, Y, p, 0)
    r, F, rp, cp = run_pluq(env, A, p, lt)
    _, _, _, _, r_oracle = orc.pluq(A, p)
    assert r == r_oracle
    check_factors(orc, A, p, r, F, rp, cp)
