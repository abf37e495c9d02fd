"""GPU parity of the bit-packed GF(2) path (fm_gf2_pack / fm_gf2_unpack /
fm_gf2_gemm) against the oracle. Bit work: every comparison is exact."""
import numpy as np
import pytest

import fm_inputs
from gpu_util import lib_and_device, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


class Gf2Matrix:
    """A device bit-packed Morton-hybrid matrix (T' = 32) owned by a torch tensor."""

    def __init__(self, fm, dev, lg, words=None):
        import torch
        self.n, self.lg = 32 << lg, lg
        self.t = torch.zeros(self.n * self.n // 32, dtype=torch.int32, device=dev)
        if words is not None:
            self.t.copy_(to_dev(words, dev))
        self.m = fm.gf2_matrix(self.t, lg)
        self.fm = fm

    def words(self) -> np.ndarray:
        return to_host(self.t)

    def sub(self, row0, col0, rows, cols):
        return self.fm.gf2_sub(self.m, row0, col0, rows, cols)


def lg_for(n):
    lg = 0
    while (32 << lg) < n:
        lg += 1
    return lg


@pytest.mark.parametrize("rows,cols,lg,ld_pad", [(64, 64, 1, 0), (70, 33, 2, 0), (1, 1, 0, 0),
                                                  (128, 100, 2, 3), (1000, 777, 5, 1), (256, 256, 3, 4)])
def test_pack_unpack_against_oracle(env, orc, rows, cols, lg, ld_pad):
    import torch
    fm, dev = env
    x = fm_inputs.uniform_residues(rows + cols, (rows, cols), 2)
    noisy = x + 2 * fm_inputs.uniform_residues(3, (rows, cols), 1000, 1)  # only bit 0 counts
    ld = cols + ld_pad
    src = np.zeros((rows, ld), dtype=np.uint32)
    src[:, :cols] = noisy
    G = Gf2Matrix(fm, dev, lg)
    G.t.fill_(-1)  # padding must be written as zero
    fm.fm_gf2_pack(to_dev(src, dev), rows, cols, ld, G.m)
    assert np.array_equal(G.words(), orc.gf2_pack(x, lg))
    out = torch.full((rows, ld), 7, dtype=torch.int32, device=dev)
    fm.fm_gf2_unpack(G.m, rows, cols, out, ld)
    got = to_host(out).reshape(rows, ld)
    assert np.array_equal(got[:, :cols], x)
    assert np.all(got[:, cols:] == 7)


def gf2_case(env, orc, M, N, K, offs, lgs, op, seed, options=None):
    fm, dev = env
    rC, cC, rA, cA, rB, cB = offs
    lC, lA, lB = lgs
    Cf = fm_inputs.uniform_residues(seed, (32 << lC, 32 << lC), 2, 1)
    Af = fm_inputs.uniform_residues(seed, (32 << lA, 32 << lA), 2, 2)
    Bf = fm_inputs.uniform_residues(seed, (32 << lB, 32 << lB), 2, 3)
    GC = Gf2Matrix(fm, dev, lC, orc.gf2_pack(Cf, lC))
    GA = Gf2Matrix(fm, dev, lA, orc.gf2_pack(Af, lA))
    GB = Gf2Matrix(fm, dev, lB, orc.gf2_pack(Bf, lB))
    fm.fm_gf2_gemm(GC.sub(rC, cC, M, N), GA.sub(rA, cA, M, K), GB.sub(rB, cB, K, N), op, options)
    assert fm.fm_get_last_device_status() == 0
    got = orc.gf2_unpack(GC.words(), lC, GC.n, GC.n)
    want = Cf.copy()
    want[rC:rC + M, cC:cC + N] = orc.gemm_modp(Cf[rC:rC + M, cC:cC + N], Af[rA:rA + M, cA:cA + K],
                                               Bf[rB:rB + K, cB:cB + N], 2, op)
    return got, want


CASES = [
    # (M, N, K, offsets (rC, cC, rA, cA, rB, cB), log2 grids)
    (256, 512, 384, (0, 0, 0, 0, 0, 0), (4, 4, 4)),
    (300, 520, 1000, (13, 70, 5, 33, 100, 3), (5, 6, 6)),
    (1, 1, 1, (0, 0, 0, 0, 0, 0), (0, 0, 0)),
    (1, 1, 1, (31, 31, 17, 5, 9, 30), (0, 0, 0)),
    (129, 257, 65, (64, 0, 0, 64, 64, 0), (4, 4, 4)),
    (17, 300, 3, (31, 1, 2, 30, 0, 5), (4, 4, 4)),
    (40, 33, 2000, (7, 31, 11, 13, 17, 19), (1, 6, 6)),
    (600, 700, 129, (100, 290, 0, 127, 1, 3), (5, 5, 5)),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("pair", [0, 1])
def test_gf2_gemm_parity(env, orc, case, pair):
    # full compare of C: the sub-matrix and every bit around it, including the
    # bits that share a word with its first and last columns; single CTAs on
    # 128 x 256 tiles and CTA pairs on 256 x 256 tiles
    M, N, K, offs, lgs = case
    options = env[0].opts(cta_pair=pair)
    for op in (0, 1, 2):
        got, want = gf2_case(env, orc, M, N, K, offs, lgs, op, seed=M + N + K + op, options=options)
        assert np.array_equal(got, want), op


def test_gf2_a_and_b_share_a_matrix(env, orc):
    # A and B inside one matrix (overlapping is allowed for the operands), C elsewhere
    fm, dev = env
    X = fm_inputs.uniform_residues(9, (256, 256), 2)
    C0 = fm_inputs.uniform_residues(10, (256, 256), 2)
    GX = Gf2Matrix(fm, dev, 3, orc.gf2_pack(X, 3))
    GC = Gf2Matrix(fm, dev, 3, orc.gf2_pack(C0, 3))
    fm.fm_gf2_gemm(GC.sub(3, 5, 200, 150), GX.sub(1, 2, 200, 170), GX.sub(50, 60, 170, 150), 1)
    want = C0.copy()
    want[3:203, 5:155] = orc.gemm_modp(C0[3:203, 5:155], X[1:201, 2:172], X[50:220, 60:210], 2, 1)
    assert np.array_equal(orc.gf2_unpack(GC.words(), 3, 256, 256), want)


def test_gf2_k0_and_empty(env, orc):
    fm, dev = env
    C0 = fm_inputs.uniform_residues(11, (128, 128), 2)
    A = Gf2Matrix(fm, dev, 2)
    for op in (0, 1):
        GC = Gf2Matrix(fm, dev, 2, orc.gf2_pack(C0, 2))
        fm.fm_gf2_gemm(GC.sub(5, 9, 50, 70), A.sub(0, 0, 50, 0), A.sub(0, 0, 0, 70), op)
        want = C0.copy()
        if op == 0:
            want[5:55, 9:79] = 0
        assert np.array_equal(orc.gf2_unpack(GC.words(), 2, 128, 128), want)
    GC = Gf2Matrix(fm, dev, 2, orc.gf2_pack(C0, 2))
    fm.fm_gf2_gemm(GC.sub(5, 9, 0, 70), A.sub(0, 0, 0, 10), A.sub(0, 0, 10, 70), 0)
    assert np.array_equal(orc.gf2_unpack(GC.words(), 2, 128, 128), C0)


def test_gf2_argument_errors(env):
    fm, dev = env
    G = Gf2Matrix(fm, dev, 2)
    H = Gf2Matrix(fm, dev, 2)
    with pytest.raises(fm.FmError):   # C overlaps A
        fm.fm_gf2_gemm(G.sub(0, 0, 40, 40), G.sub(30, 30, 40, 10), H.sub(0, 0, 10, 40))
    with pytest.raises(fm.FmError):   # shapes disagree
        fm.fm_gf2_gemm(G.sub(0, 0, 40, 40), H.sub(0, 0, 41, 10), H.sub(0, 0, 10, 40))
    with pytest.raises(fm.FmError):   # outside the matrix
        fm.fm_gf2_gemm(G.sub(100, 0, 40, 40), H.sub(0, 0, 40, 10), H.sub(0, 0, 10, 40))
    with pytest.raises(fm.FmError):   # bad op
        fm.fm_gf2_gemm(G.sub(0, 0, 4, 4), H.sub(0, 0, 4, 4), H.sub(4, 4, 4, 4), 3)
    # C and A in one matrix but disjoint (they may share words): allowed
    fm.fm_gf2_gemm(G.sub(0, 0, 40, 20), G.sub(0, 20, 40, 10), H.sub(0, 0, 10, 20))
    assert fm.fm_gf2_workspace_size(4096, 4096, 4096) == 32 * 32 * 16384 + 16 * 32 * 32768


def test_gf2_paper_workload_random_subproducts(env, orc):
    # the experiments' workload (Sec. 2.2, "Performance Analysis"): products of
    # random sub-matrices of three 2048 x 2048 Morton-hybrid matrices over GF(2)
    # with T' = 32; 12 of them, each checked on 400 sampled entries and by 16
    # Freivalds trials (a wrong product passes one with probability <= 1/2)
    fm, dev = env
    lg = 6
    n = 2048
    Cf = fm_inputs.uniform_residues(21, (n, n), 2, 1)
    Af = fm_inputs.uniform_residues(21, (n, n), 2, 2)
    Bf = fm_inputs.uniform_residues(21, (n, n), 2, 3)
    GA = Gf2Matrix(fm, dev, lg, orc.gf2_pack(Af, lg))
    GB = Gf2Matrix(fm, dev, lg, orc.gf2_pack(Bf, lg))
    for t, rect in enumerate(fm_inputs.sub_rectangles(468, 12, n)):
        M, N, K, rC, cC, rA, cA, rB, cB = (int(x) for x in rect)
        GC = Gf2Matrix(fm, dev, lg, orc.gf2_pack(Cf, lg))
        fm.fm_gf2_gemm(GC.sub(rC, cC, M, N), GA.sub(rA, cA, M, K), GB.sub(rB, cB, K, N), 1)
        got = orc.gf2_unpack(GC.words(), lg, n, n)
        # outside the sub-matrix nothing changed
        mask = np.ones((n, n), dtype=bool)
        mask[rC:rC + M, cC:cC + N] = False
        assert np.array_equal(got[mask], Cf[mask]), t
        Cin, Cout = Cf[rC:rC + M, cC:cC + N], got[rC:rC + M, cC:cC + N]
        A, B = Af[rA:rA + M, cA:cA + K], Bf[rB:rB + K, cB:cB + N]
        ij = np.stack([fm_inputs.integers(t, 400, 0, M - 1, 1), fm_inputs.integers(t, 400, 0, N - 1, 2)], 1)
        assert np.array_equal(Cout[ij[:, 0], ij[:, 1]], orc.gemm_modp_entries(Cin, A, B, 2, 1, ij)), t
        assert orc.freivalds(Cout, Cin, A, B, 2, 1, trials=16, seed=t), t


def test_gf2_8192(env, orc):
    # n = 8192 over GF(2): 3000 sampled entries against the oracle and 24 Freivalds trials
    fm, dev = env
    n, lg = 8192, 8
    A = fm_inputs.uniform_residues(31, (n, n), 2, 1)
    B = fm_inputs.uniform_residues(31, (n, n), 2, 2)
    C = fm_inputs.uniform_residues(31, (n, n), 2, 3)
    GA = Gf2Matrix(fm, dev, lg, orc.gf2_pack(A, lg))
    GB = Gf2Matrix(fm, dev, lg, orc.gf2_pack(B, lg))
    ij = np.stack([fm_inputs.integers(7, 3000, 0, n - 1, 1), fm_inputs.integers(7, 3000, 0, n - 1, 2)], 1)
    want = orc.gemm_modp_entries(C, A, B, 2, 1, ij)
    for pair in (0, 1):
        GC = Gf2Matrix(fm, dev, lg, orc.gf2_pack(C, lg))
        fm.fm_gf2_gemm(GC.sub(0, 0, n, n), GA.sub(0, 0, n, n), GB.sub(0, 0, n, n), 1, fm.opts(cta_pair=pair))
        assert fm.fm_get_last_device_status() == 0
        got = orc.gf2_unpack(GC.words(), lg, n, n)
        assert np.array_equal(got[ij[:, 0], ij[:, 1]], want), pair
        assert orc.freivalds(got, C, A, B, 2, 1, trials=24, seed=3 + pair), pair


def _gf2_call(fm, C, A, B, op):
    call = fm.fm_gf2_call()
    call.C, call.A, call.B = C, A, B
    call.op = op
    return call


def test_gf2_plan_matches_per_call_and_oracle(env, orc):
    # a batch of random sub-matrix products (the experiments' workload) as one
    # plan; C regions of different calls are disjoint rows but share words
    fm, dev = env
    lg, n = 5, 1024
    Cf = fm_inputs.uniform_residues(41, (n, n), 2, 1)
    Af = fm_inputs.uniform_residues(41, (n, n), 2, 2)
    Bf = fm_inputs.uniform_residues(41, (n, n), 2, 3)
    GA = Gf2Matrix(fm, dev, lg, orc.gf2_pack(Af, lg))
    GB = Gf2Matrix(fm, dev, lg, orc.gf2_pack(Bf, lg))
    GC = Gf2Matrix(fm, dev, lg, orc.gf2_pack(Cf, lg))
    rects = fm_inputs.sub_rectangles(77, 30, 300)
    calls, meta = [], []
    for t, r in enumerate(rects):
        M, N, K, _, cC, rA, cA, rB, cB = (int(x) for x in r)
        M = min(M, 30)           # 30 bands of 30 rows: disjoint C regions
        rC = 32 * t + 1          # ... starting at odd rows, columns anywhere
        op = t % 3
        calls.append(_gf2_call(fm, GC.sub(rC, cC, M, N), GA.sub(rA, cA, M, K), GB.sub(rB, cB, K, N), op))
        meta.append((M, N, K, rC, cC, rA, cA, rB, cB, op))
    calls.append(_gf2_call(fm, GC.sub(980, 3, 20, 50), GA.sub(0, 0, 20, 0), GB.sub(0, 0, 0, 50), 0))  # K = 0
    meta.append((20, 50, 0, 980, 3, 0, 0, 0, 0, 0))
    plan = fm.fm_gf2_plan_create(calls)
    assert plan.work_items > 0
    plan.run()
    assert fm.fm_get_last_device_status() == 0
    got = orc.gf2_unpack(GC.words(), lg, n, n)
    want = Cf.copy()
    for (M, N, K, rC, cC, rA, cA, rB, cB, op) in meta:
        want[rC:rC + M, cC:cC + N] = orc.gemm_modp(want[rC:rC + M, cC:cC + N], Af[rA:rA + M, cA:cA + K],
                                                   Bf[rB:rB + K, cB:cB + N], 2, op)
    assert np.array_equal(got, want)
    # one fm_gf2_gemm per call from the same start: the same bits
    GC2 = Gf2Matrix(fm, dev, lg, orc.gf2_pack(Cf, lg))
    for c in calls:
        C = c.C
        fm.fm_gf2_gemm(GC2.sub(C.row0, C.col0, C.rows, C.cols), c.A, c.B, c.op)
    assert np.array_equal(GC2.words(), GC.words())
    plan.close()


def test_gf2_plan_graph_replay(env, orc):
    import torch
    fm, dev = env
    lg, n = 4, 512
    Cf = fm_inputs.uniform_residues(43, (n, n), 2, 1)
    Af = fm_inputs.uniform_residues(43, (n, n), 2, 2)
    GA = Gf2Matrix(fm, dev, lg, orc.gf2_pack(Af, lg))
    GC = Gf2Matrix(fm, dev, lg, orc.gf2_pack(Cf, lg))
    calls = [_gf2_call(fm, GC.sub(100 * t, 7 * t, 90, 200), GA.sub(3 * t, 5, 90, 300),
                       GA.sub(11, 13 * t, 300, 200), 1) for t in range(5)]
    plan = fm.fm_gf2_plan_create(calls)
    fm.fm_get_last_device_status()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    torch.cuda.synchronize()
    g.replay()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    want = Cf.copy()
    for t in range(5):   # three additions of the same product: C + A B over GF(2)
        blk = want[100 * t:100 * t + 90, 7 * t:7 * t + 200]
        want[100 * t:100 * t + 90, 7 * t:7 * t + 200] = orc.gemm_modp(
            blk, Af[3 * t:3 * t + 90, 5:305], Af[11:311, 13 * t:13 * t + 200], 2, 1)
    assert np.array_equal(orc.gf2_unpack(GC.words(), lg, n, n), want)
    plan.close()


def test_gf2_plan_errors(env):
    fm, dev = env
    G = Gf2Matrix(fm, dev, 2)
    H = Gf2Matrix(fm, dev, 2)
    bad = _gf2_call(fm, G.sub(0, 0, 40, 40), G.sub(30, 30, 40, 10), H.sub(0, 0, 10, 40), 0)
    with pytest.raises(fm.FmError):
        fm.fm_gf2_plan_create([bad])
    ok = _gf2_call(fm, G.sub(0, 0, 40, 40), H.sub(0, 0, 40, 10), H.sub(0, 0, 10, 40), 0)
    with pytest.raises(fm.FmError):
        fm.fm_gf2_plan_create([ok], fm.opts(cta_pair=1))
    empty = fm.fm_gf2_plan_create([])
    assert empty.work_items == 0
    empty.run()
    empty.close()
