"""GPU parity of C <- C op A*B mod p (plain, DFMA and tensor-core limb forms)
against the oracle. Integer work: every comparison is bit-exact."""
import numpy as np
import pytest

import fm_inputs
from gpu_util import MortonMatrix, grid_for, lib_and_device, to_dev, to_host

pytestmark = pytest.mark.gpu

P16, P31 = 65521, 2147483647


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def run_case(env, orc, p, op, algo, M, N, K, offs, lts, seed, options=None):
    """Random full matrices, the product on the sub-matrices at offs, full
    comparison of the whole C matrix (nothing outside the part may change)."""
    fm, dev = env
    rC, cC, rA, cA, rB, cB = offs
    ltC, ltA, ltB = lts
    lgC = grid_for(rC + M, cC + N, ltC)
    lgA = grid_for(rA + M, cA + K, ltA)
    lgB = grid_for(rB + K, cB + N, ltB)
    nC, nA, nB = (1 << lgC) << ltC, (1 << lgA) << ltA, (1 << lgB) << ltB
    Cf = fm_inputs.uniform_residues(seed, (nC, nC), p, 1)
    Af = fm_inputs.uniform_residues(seed, (nA, nA), p, 2)
    Bf = fm_inputs.uniform_residues(seed, (nB, nB), p, 3)
    MC = MortonMatrix(fm, dev, lgC, ltC, fill=Cf)
    MA = MortonMatrix(fm, dev, lgA, ltA, fill=Af)
    MB = MortonMatrix(fm, dev, lgB, ltB, fill=Bf)
    fm.fm_gemm_modp(MC.sub(rC, cC, M, N), MA.sub(rA, cA, M, K), MB.sub(rB, cB, K, N), p, op, algo,
                    options)
    got = MC.read()
    assert fm.fm_get_last_device_status() == 0
    want = Cf.copy()
    want[rC:rC + M, cC:cC + N] = orc.gemm_modp(Cf[rC:rC + M, cC:cC + N], Af[rA:rA + M, cA:cA + K],
                                               Bf[rB:rB + K, cB:cB + N], p, op)
    return got, want


CASES = [
    # (M, N, K, offsets (rC, cC, rA, cA, rB, cB))
    (300, 520, 1000, (0, 0, 0, 0, 0, 0)),
    (300, 520, 1000, (13, 70, 5, 33, 100, 3)),
    (1, 1, 1, (0, 0, 0, 0, 0, 0)),
    (129, 257, 65, (64, 0, 0, 64, 64, 0)),
    (64, 64, 2000, (7, 9, 11, 13, 17, 19)),
    (17, 300, 3, (31, 1, 2, 30, 0, 5)),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("lt", [5, 6])
def test_plain_parity(env, orc, case, lt):
    M, N, K, offs = case
    for p, op in ((P16, 2), (P31, 1), (2, 0), (257, 2)):
        got, want = run_case(env, orc, p, op, env[0].FM_ALGO_PLAIN, M, N, K, offs, (lt, lt, lt),
                             seed=M + N + K + p)
        assert np.array_equal(got, want), (p, op)


@pytest.mark.parametrize("case", CASES[:4])
def test_dfma_parity(env, orc, case):
    M, N, K, offs = case
    for p, op in ((P16, 2), (3, 1)):
        got, want = run_case(env, orc, p, op, env[0].FM_ALGO_DFMA, M, N, K, offs, (6, 6, 6), seed=K)
        assert np.array_equal(got, want), (p, op)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("p", [2, 251, 257, P16, 65534, 65537, 1000003, P31])
def test_limb_parity(env, orc, case, p):
    M, N, K, offs = case
    for op, lts in ((2, (6, 6, 6)), (0, (7, 4, 5)), (1, (5, 7, 3))):
        got, want = run_case(env, orc, p, op, env[0].FM_ALGO_LIMB_TC, M, N, K, offs, lts,
                             seed=M * 3 + p % 1000 + op)
        assert np.array_equal(got, want), (p, op, lts)


@pytest.mark.parametrize("k_chunk,block_n,no_kara,pair", [
    (64, 0, 0, 0), (512, 0, 0, 0), (960, 0, 0, 0), (0, 128, 0, 0), (320, 128, 0, 0),
    (0, 0, 1, 0), (192, 128, 1, 0), (0, 256, 0, 1), (960, 256, 1, 1), (64, 256, 0, 1)])
def test_limb_chunk_and_tile_options(env, orc, k_chunk, block_n, no_kara, pair):
    fm = env[0]
    for p in (P16, 257):
        got, want = run_case(env, orc, p, 2, fm.FM_ALGO_LIMB_TC, 300, 520, 3000, (0, 5, 3, 0, 0, 9),
                             (6, 6, 6), seed=4, options=fm.opts(k_chunk, block_n, no_kara, pair))
        assert np.array_equal(got, want), p


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (129, 256, 960), (300, 520, 1000),
                                   (2560, 2048, 128), (1000, 3000, 200)])
def test_limb_cta_pair_and_single_cta(env, orc, M, N, K):
    # 256 x 256 tiles on CTA pairs against 128 x 256 tiles on single CTAs: an
    # odd number of 128-row blocks (the pair's second half past M), one tile,
    # and more pair tiles than pairs resident on the device (the persistent walk)
    fm = env[0]
    for p in (P16, 251, 2):
        for pair in (-1, 1):
            got, want = run_case(env, orc, p, 2, fm.FM_ALGO_LIMB_TC, M, N, K, (0, 3, 5, 0, 0, 7),
                                 (7, 7, 7), seed=M + N + p, options=fm.opts(0, 256, 0, pair))
            assert np.array_equal(got, want), (p, pair)


@pytest.mark.parametrize("M,N,K", [(300, 520, 4096), (300, 520, 4097), (2560, 2048, 128), (129, 1000, 64)])
def test_limb_fold_two_ctas_per_sm(env, orc, M, N, K):
    # fold form on 128-wide tiles: two CTAs per SM up to K = 4096, one beyond;
    # both sides of that bound, more tiles than the 2 x 152 resident CTAs, and
    # a single row block
    fm = env[0]
    for p, op in ((P16, 2), (257, 0), (2, 1)):
        got, want = run_case(env, orc, p, op, fm.FM_ALGO_LIMB_TC, M, N, K, (3, 0, 0, 5, 7, 0),
                             (7, 6, 7), seed=K + p, options=fm.opts(0, 128, 0, -1))
        assert np.array_equal(got, want), (p, op)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (129, 130, 1000), (300, 520, 1000),
                                   (2560, 2048, 128), (1000, 3000, 200), (513, 257, 2100)])
def test_limb_residue_cta_pair_and_single_cta(env, orc, M, N, K):
    # residue form (p >= 2^16 or even p): 256 x 128 tiles on CTA pairs against
    # 128 x 128 tiles on single CTAs; one tile whose second half lies past M,
    # ragged columns, more pair tiles than pairs resident on the device, and
    # K spanning several chunks of every product
    fm = env[0]
    for p, op in ((P31, 2), (65537, 0), (65534, 1), (1000003, 2)):
        for pair in (-1, 1):
            got, want = run_case(env, orc, p, op, fm.FM_ALGO_LIMB_TC, M, N, K, (0, 3, 5, 0, 0, 7),
                                 (7, 6, 7), seed=M + N + p % 997 + pair,
                                 options=fm.opts(0, 128, 0, pair))
            assert np.array_equal(got, want), (p, op, pair)


@pytest.mark.parametrize("pair", [-1, 1])
def test_limb_residue_sum_refresh(env, orc, pair):
    # With 64-wide chunks a product at K = 8000 has 125 chunks: its int32 sum S
    # is folded into the residue after chunk 119 and restarted at chunk 120
    # (120 chunks of at most 2^24 stay inside int32). Random inputs, and the
    # extremes whose every chunk sums to exactly 2^24.
    fm = env[0]
    o = fm.opts(64, 128, 0, pair)
    got, want = run_case(env, orc, P31, 2, fm.FM_ALGO_LIMB_TC, 300, 200, 8000, (1, 2, 3, 4, 5, 6),
                         (6, 6, 6), seed=120 + pair, options=o)
    assert np.array_equal(got, want)
    lo = 8355712  # digits (-128, -128, -128, 1)
    hi = 127 * (1 + 256 + 65536)  # digits (127, 127, 127, 0): negative sums against lo
    for a, b in ((P31 - 128, P31 - 128), (lo, lo), (lo, hi), (P31 - 128, 127)):
        _constant_case(env, orc, P31, a, b, 8000, fm.FM_ALGO_LIMB_TC, o)


def test_limb_rejects_unsafe_chunk(env):
    fm, dev = env
    M = MortonMatrix(fm, dev, 1, 7)
    A = MortonMatrix(fm, dev, 1, 7)
    with pytest.raises(fm.FmError):   # 1024 > the exact bound 960 when folding p = 65521
        fm.fm_gemm_modp(M.sub(0, 0, 64, 64), A.sub(0, 0, 64, 64), A.sub(0, 0, 64, 64), P16, 0,
                        fm.FM_ALGO_LIMB_TC, fm.opts(1024, 0))
    with pytest.raises(fm.FmError):   # CTA pairs: 256-wide tiles in the fold form
        fm.fm_gemm_modp(M.sub(0, 0, 64, 64), A.sub(0, 0, 64, 64), A.sub(0, 0, 64, 64), P16, 0,
                        fm.FM_ALGO_LIMB_TC, fm.opts(0, 128, 0, 1))
    with pytest.raises(fm.FmError):   # and 128-wide tiles in the residue form
        fm.fm_gemm_modp(M.sub(0, 0, 64, 64), A.sub(0, 0, 64, 64), A.sub(0, 0, 64, 64), P31, 0,
                        fm.FM_ALGO_LIMB_TC, fm.opts(0, 256, 0, 1))


def _constant_case(env, orc, p, a, b, K, algo, options=None):
    fm, dev = env
    M, N = 256, 512
    lt = 7
    lg = grid_for(max(M, K), max(N, K), lt)
    MA = MortonMatrix(fm, dev, lg, lt, fill=np.full((M, K), a, dtype=np.uint32))
    MB = MortonMatrix(fm, dev, lg, lt, fill=np.full((K, N), b, dtype=np.uint32))
    MC = MortonMatrix(fm, dev, grid_for(M, N, lt), lt)
    fm.fm_gemm_modp(MC.sub(0, 0, M, N), MA.sub(0, 0, M, K), MB.sub(0, 0, K, N), p, 0, algo, options)
    got = MC.read(M, N)
    closed = (K * a % p) * b % p
    assert np.all(got == closed), (p, a, b, K)
    assert fm.fm_get_last_device_status() == 0


@pytest.mark.parametrize("K", [64, 960, 961, 1024, 2048, 8192])
def test_limb_accumulator_extremes_p16(env, orc, K):
    # Inputs whose limbs are all -128 make every limb product +2^14, the largest
    # magnitude; a chunk of 960 with a folded residue reaches 960*2^14 + p - 1,
    # just under 2^24. 65393 = p - 128 has limbs (-128, 0); 32753 = p - 32768
    # has limbs (0, -128); 127 has limbs (127, 0). 32881 = p - 32640 has limbs
    # (-128, -127): its Karatsuba middle term is (-255)^2 = 65025, and a 256-term
    # middle chunk with its carried value reaches 16,646,400 + |carry| < 2^24.
    fm = env[0]
    for a, b in ((65393, 65393), (32753, 32753), (65393, 32753), (127, 65393), (32639, 32753),
                 (32881, 32881), (32881, 32639), (32639, 32639)):
        _constant_case(env, orc, P16, a, b, K, fm.FM_ALGO_LIMB_TC)


@pytest.mark.parametrize("K", [1024, 2048, 4096])
def test_limb_accumulator_extremes_p31(env, orc, K):
    # p = 2^31 - 1, chunk 1024 without folding: all limbs -128 sum to exactly
    # 2^24 per chunk. x = p - 128 * 256^t (t < 3) has limb t equal to -128; the
    # top limb of a representative lies in [-1, 127], so 127 * 256^3 is its
    # extreme. On single CTAs and on CTA pairs.
    fm = env[0]
    extremes = [P31 - 128 * 256 ** t for t in range(3)] + [127 * 256 ** 3]
    for o in (fm.opts(0, 128, 0, -1), fm.opts(0, 128, 0, 1)):
        for a in extremes:
            _constant_case(env, orc, P31, a, a, K, fm.FM_ALGO_LIMB_TC, o)
        _constant_case(env, orc, P31, extremes[0], extremes[3], K, fm.FM_ALGO_LIMB_TC, o)


@pytest.mark.parametrize("K", [256, 512, 1024, 2048])
@pytest.mark.parametrize("p", [P31, 1000003, 65537])
def test_limb_karatsuba_pair_extremes(env, orc, K, p):
    # The residue form multiplies the digit sums d_i + d_j of every pair of
    # limbs in chunks of 256 terms. Inputs whose pair digits are both -128 make
    # those terms (-256)^2 = 2^16, so a 256-term chunk sums to exactly 2^24:
    # x = 256^3 - 128 (1 + 256 + 256^2) = 8355712 has digits (-128, -128, -128, 1)
    # for w = 4; x = 256^2 - 128 (1 + 256) = 32640 has digits (-128, -128, 1) for
    # w = 3. Mixed with the +127 extremes (digit sums 254) as well.
    fm = env[0]
    w = 4 if p > (1 << 24) else 3
    lo = 8355712 if w == 4 else 32640
    hi = 127 * (1 + 256 + 65536) if w == 4 else 127 * 257
    for o in (fm.opts(0, 128, 0, -1), fm.opts(0, 128, 0, 1)):
        for a, b in ((lo, lo), (lo, hi), (hi, hi)):
            _constant_case(env, orc, p, a, b, K, fm.FM_ALGO_LIMB_TC, o)


def test_empty_and_degenerate(env, orc):
    fm, dev = env
    C = MortonMatrix(fm, dev, 2, 5, fill=fm_inputs.uniform_residues(1, (128, 128), P16))
    A = MortonMatrix(fm, dev, 2, 5, fill=fm_inputs.uniform_residues(2, (128, 128), P16))
    before = C.read()
    for algo in (fm.FM_ALGO_PLAIN, fm.FM_ALGO_LIMB_TC, fm.FM_ALGO_DFMA):
        fm.fm_gemm_modp(C.sub(3, 4, 20, 30), A.sub(0, 0, 20, 0), A.sub(0, 0, 0, 30), P16, 2, algo)
        fm.fm_gemm_modp(C.sub(3, 4, 0, 30), A.sub(0, 0, 0, 7), A.sub(0, 0, 7, 30), P16, 2, algo)
    assert np.array_equal(C.read(), before)
    fm.fm_gemm_modp(C.sub(3, 4, 20, 30), A.sub(0, 0, 20, 0), A.sub(0, 0, 0, 30), P16, 0, 1)
    after = C.read()
    expect = before.copy()
    expect[3:23, 4:34] = 0
    assert np.array_equal(after, expect)


def test_argument_errors(env):
    fm, dev = env
    C = MortonMatrix(fm, dev, 2, 5)
    A = MortonMatrix(fm, dev, 2, 6)
    cases = [
        (C.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), 1 << 31, 0, 0),   # modulus
        (C.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), 1, 0, 0),         # modulus
        (C.sub(0, 0, 8, 8), A.sub(0, 0, 8, 9), A.sub(0, 0, 8, 8), P16, 0, 0),       # inner dims
        (C.sub(0, 0, 8, 8), C.sub(4, 4, 8, 8), A.sub(0, 0, 8, 8), P16, 0, 0),       # overlap
        (C.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), P16, 0, 1),       # T' differ
        (C.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), P16, 7, 0),       # op
        (C.sub(120, 0, 9, 8), A.sub(0, 0, 9, 8), A.sub(0, 0, 8, 8), P16, 0, 0),     # outside
    ]
    C6 = MortonMatrix(fm, dev, 2, 6)
    cases.append((C6.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), A.sub(0, 0, 8, 8), P31, 0, 4))  # dfma bound
    for c, a, b, p, op, algo in cases:
        with pytest.raises(fm.FmError):
            fm.fm_gemm_modp(c, a, b, p, op, algo)


# ---- BASELINE workloads at full size ---------------------------------------
def _dense(fm, dev, x, lt):
    n = x.shape[0]
    lg = grid_for(n, n, lt)
    return MortonMatrix(fm, dev, lg, lt, fill=x)


def test_config1_256_plain(env, orc):
    # 256^3, p = 65521, T' = 32 (8 x 8 tiles), plain CUDA-core path, C = A*B
    fm, dev = env
    A = fm_inputs.uniform_residues(0, (256, 256), P16, 1)
    B = fm_inputs.uniform_residues(0, (256, 256), P16, 2)
    MA, MB = _dense(fm, dev, A, 5), _dense(fm, dev, B, 5)
    MC = MortonMatrix(fm, dev, 3, 5)
    fm.fm_gemm_modp(MC.sub(0, 0, 256, 256), MA.sub(0, 0, 256, 256), MB.sub(0, 0, 256, 256), P16, 0,
                    fm.FM_ALGO_PLAIN)
    assert np.array_equal(MC.read(), orc.gemm_modp(None, A, B, P16, 0))


def test_config2_schur_update_plain(env, orc):
    # C (3000 x 2200) -= A (3000 x 1700) * B (1700 x 2200) mod 65521, T' = 64,
    # row-major inputs permuted and converted to Morton-hybrid on the device.
    fm, dev = env
    M, K, N = 3000, 1700, 2200
    A = fm_inputs.uniform_residues(2, (M, K), P16, 1)
    B = fm_inputs.uniform_residues(2, (K, N), P16, 2)
    C = fm_inputs.uniform_residues(2, (M, N), P16, 3)
    rpA, cpA = fm_inputs.permutation(2, M, 4), fm_inputs.permutation(2, K, 5)
    rpB, cpB = fm_inputs.permutation(2, K, 6), fm_inputs.permutation(2, N, 7)
    MA, MB, MC = (MortonMatrix(fm, dev, 6, 6) for _ in range(3))
    fm.fm_layout_to_morton_permuted(to_dev(A, dev), M, K, K, to_dev(rpA, dev), to_dev(cpA, dev), MA.m)
    fm.fm_layout_to_morton_permuted(to_dev(B, dev), K, N, N, to_dev(rpB, dev), to_dev(cpB, dev), MB.m)
    fm.fm_layout_to_morton(to_dev(C, dev), M, N, N, MC.m)
    for algo in (fm.FM_ALGO_PLAIN, fm.FM_ALGO_LIMB_TC):
        MC2 = MortonMatrix(fm, dev, 6, 6)
        MC2.t.copy_(MC.t)
        fm.fm_gemm_modp(MC2.sub(0, 0, M, N), MA.sub(0, 0, M, K), MB.sub(0, 0, K, N), P16, 2, algo)
        got = MC2.read(M, N)
        want = orc.gemm_modp(C, orc.permute(A, rpA, cpA), orc.permute(B, rpB, cpB), P16, 2)
        assert np.array_equal(got, want), algo


def test_config3_8192_limb_plain_dfma(env, orc):
    # 8192^3, p = 65521: the tensor-core limb form against the oracle's full
    # product, every entry (about 20 s on 16 host cores), plus two Freivalds
    # trials; the plain and DFMA forms bit-identical to it.
    fm, dev = env
    n = 8192
    A = fm_inputs.uniform_residues(3, (n, n), P16, 1)
    B = fm_inputs.uniform_residues(3, (n, n), P16, 2)
    MA, MB = _dense(fm, dev, A, 7), _dense(fm, dev, B, 7)
    outs = {}
    for algo in (fm.FM_ALGO_LIMB_TC, fm.FM_ALGO_PLAIN, fm.FM_ALGO_DFMA):
        lt = 7 if algo == fm.FM_ALGO_LIMB_TC else 6
        if algo != fm.FM_ALGO_LIMB_TC and MA.lt != 6:
            MA, MB = _dense(fm, dev, A, 6), _dense(fm, dev, B, 6)
        MC = MortonMatrix(fm, dev, grid_for(n, n, lt), lt)
        fm.fm_gemm_modp(MC.sub(0, 0, n, n), MA.sub(0, 0, n, n), MB.sub(0, 0, n, n), P16, 0, algo)
        outs[algo] = MC.read()
        assert fm.fm_get_last_device_status() == 0
    limb = outs[fm.FM_ALGO_LIMB_TC]
    assert np.array_equal(limb, orc.gemm_modp(None, A, B, P16, 0))
    assert orc.freivalds(limb, None, A, B, P16, 0, trials=2)
    assert np.array_equal(outs[fm.FM_ALGO_PLAIN], limb)
    assert np.array_equal(outs[fm.FM_ALGO_DFMA], limb)


def test_config4_4096_p31(env, orc):
    # 4096^3, p = 2^31 - 1, 4 limbs: the oracle's full product, every entry,
    # two Freivalds trials, and the plain (96-bit accumulation) form
    # bit-identical.
    fm, dev = env
    n = 4096
    A = fm_inputs.uniform_residues(4, (n, n), P31, 1)
    B = fm_inputs.uniform_residues(4, (n, n), P31, 2)
    C = fm_inputs.uniform_residues(4, (n, n), P31, 3)
    outs = {}
    for algo, lt in ((fm.FM_ALGO_LIMB_TC, 7), (fm.FM_ALGO_PLAIN, 6)):
        MA, MB, MC = _dense(fm, dev, A, lt), _dense(fm, dev, B, lt), _dense(fm, dev, C, lt)
        fm.fm_gemm_modp(MC.sub(0, 0, n, n), MA.sub(0, 0, n, n), MB.sub(0, 0, n, n), P31, 2, algo)
        outs[algo] = MC.read()
        assert fm.fm_get_last_device_status() == 0
    limb = outs[fm.FM_ALGO_LIMB_TC]
    assert np.array_equal(limb, orc.gemm_modp(C, A, B, P31, 2))
    assert orc.freivalds(limb, C, A, B, P31, 2, trials=2)
    assert np.array_equal(outs[fm.FM_ALGO_PLAIN], limb)
