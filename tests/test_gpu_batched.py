"""GPU parity of the batching form: many uneven calls in one persistent launch
(Sec. 2.2, Prop. on work and span: the base-case products are independent)."""
import numpy as np
import pytest

import fm_inputs
from gpu_util import MortonMatrix, lib_and_device

pytestmark = pytest.mark.gpu

P16 = 65521


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def make_batch(fm, dev, count, seed, lt=6, lo=32, hi=512, block=512, big=4096):
    """count calls with M, N, K uniform in [lo, hi]; call c writes its own
    block x block cell of C (disjoint), A and B parts are random rectangles of
    shared matrices (reads may overlap)."""
    cells = big // block
    assert count <= cells * cells
    lg = 0
    while (1 << lg) << lt < big:
        lg += 1
    Cf = fm_inputs.uniform_residues(seed, (big, big), P16, 1)
    Af = fm_inputs.uniform_residues(seed, (big, big), P16, 2)
    Bf = fm_inputs.uniform_residues(seed, (big, big), P16, 3)
    MC = MortonMatrix(fm, dev, lg, lt, fill=Cf)
    MA = MortonMatrix(fm, dev, lg, lt, fill=Af)
    MB = MortonMatrix(fm, dev, lg, lt, fill=Bf)
    shapes = fm_inputs.batch_shapes(seed, count, lo, hi)
    offs = fm_inputs.raw_u64(seed, 6 * count, 9).reshape(count, 6)
    calls, meta = [], []
    for c in range(count):
        M, N, K = (int(x) for x in shapes[c])
        cr, cc = (c // cells) * block, (c % cells) * block
        cr += int(offs[c, 0]) % (block - M + 1)
        cc += int(offs[c, 1]) % (block - N + 1)
        ar, ac = int(offs[c, 2]) % (big - M + 1), int(offs[c, 3]) % (big - K + 1)
        br, bc = int(offs[c, 4]) % (big - K + 1), int(offs[c, 5]) % (big - N + 1)
        op = c % 3
        call = fm.fm_gemm_call()
        call.C, call.A, call.B = MC.sub(cr, cc, M, N), MA.sub(ar, ac, M, K), MB.sub(br, bc, K, N)
        call.op = op
        calls.append(call)
        meta.append((M, N, K, cr, cc, ar, ac, br, bc, op))
    return MC, MA, MB, Cf, Af, Bf, calls, meta


def expected(orc, Cf, Af, Bf, meta, times=1, p=P16):
    want = Cf.copy()
    for (M, N, K, cr, cc, ar, ac, br, bc, op) in meta:
        blk = want[cr:cr + M, cc:cc + N]
        for _ in range(times):
            blk = orc.gemm_modp(blk, Af[ar:ar + M, ac:ac + K], Bf[br:br + K, bc:bc + N], p, op)
        want[cr:cr + M, cc:cc + N] = blk
    return want


@pytest.mark.parametrize("lt", [5, 6])
def test_batched_matches_oracle_and_per_call(env, orc, lt):
    fm, dev = env
    MC, MA, MB, Cf, Af, Bf, calls, meta = make_batch(fm, dev, 48, seed=lt, lt=lt)
    plan = fm.fm_plan_create(calls, P16, fm.FM_ALGO_PLAIN)
    assert plan.work_items > 0
    saved = MC.t.clone()
    plan.run()
    got = MC.read()
    assert fm.fm_get_last_device_status() == 0
    assert np.array_equal(got, expected(orc, Cf, Af, Bf, meta))
    # one launch per call gives the same integers
    MC.t.copy_(saved)
    for call in calls:
        fm.fm_gemm_modp(call.C, call.A, call.B, P16, call.op, fm.FM_ALGO_PLAIN)
    assert np.array_equal(MC.read(), got)
    plan.close()


def test_batched_graph_capture_and_replay(env, orc):
    import torch
    fm, dev = env
    MC, MA, MB, Cf, Af, Bf, calls, meta = make_batch(fm, dev, 16, seed=9)
    plan = fm.fm_plan_create(calls, P16, fm.FM_ALGO_AUTO)
    fm.fm_get_last_device_status()  # device status word exists before capture
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    torch.cuda.synchronize()
    assert np.array_equal(MC.read(), Cf)  # capture does not execute
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(MC.read(), expected(orc, Cf, Af, Bf, meta, times=2))
    plan.close()


def test_empty_plan_and_errors(env):
    fm, dev = env
    plan = fm.fm_plan_create([], P16)
    assert plan.work_items == 0
    plan.run()
    plan.close()
    M = MortonMatrix(fm, dev, 1, 6)
    call = fm.fm_gemm_call()
    call.C, call.A, call.B = M.sub(0, 0, 8, 8), M.sub(8, 8, 8, 8), M.sub(4, 4, 8, 8)  # overlap
    with pytest.raises(fm.FmError):
        fm.fm_plan_create([call], P16)


P31 = 2147483647


@pytest.mark.parametrize("p,opt", [(P16, {}), (P16, {"block_n": 128}), (P16, {"no_karatsuba": 1}),
                                   (P31, {}), (257, {})])
@pytest.mark.parametrize("lt", [6, 7])
def test_limb_batched_matches_oracle_and_per_call(env, orc, p, opt, lt):
    # the tensor-core form for a whole batch (2 split launches + 1 GEMM launch)
    # against the oracle and against one fm_gemm_modp call per product (inputs
    # reduced mod p when p < 65521)
    fm, dev = env
    MC, MA, MB, Cf, Af, Bf, calls, meta = make_batch(fm, dev, 40, seed=lt + p % 7, lt=lt)
    if p < P16:  # inputs must be residues mod p
        Cf, Af, Bf = Cf % p, Af % p, Bf % p
        MC.load(Cf)
        MA.load(Af)
        MB.load(Bf)
    o = fm.opts(**opt)
    plan = fm.fm_plan_create(calls, p, fm.FM_ALGO_LIMB_TC, o)
    assert plan.work_items > 0
    saved = MC.t.clone()
    plan.run()
    got = MC.read()
    assert fm.fm_get_last_device_status() == 0
    assert np.array_equal(got, expected(orc, Cf, Af, Bf, meta, p=p))
    MC.t.copy_(saved)
    for call in calls:
        fm.fm_gemm_modp(call.C, call.A, call.B, p, call.op, fm.FM_ALGO_LIMB_TC, o)
    assert np.array_equal(MC.read(), got)
    plan.close()


def test_limb_batched_with_empty_and_k0_calls(env, orc):
    # calls with K = 0 (SET zeroes C, ADD/SUB leave it) and with M or N = 0
    fm, dev = env
    MC, MA, MB, Cf, Af, Bf, calls, meta = make_batch(fm, dev, 12, seed=3, lt=6)
    extra_meta = []
    for c, (M, N, K, op) in enumerate([(40, 50, 0, 0), (30, 20, 0, 1), (0, 10, 5, 0), (10, 0, 5, 2)]):
        call = fm.fm_gemm_call()
        r0 = 3800 + 60 * c  # a free corner of C (make_batch uses cells < 12 of the 8 x 8 grid)
        call.C, call.A, call.B = MC.sub(r0, 3900, M, N), MA.sub(7, 9, M, K), MB.sub(11, 13, K, N)
        call.op = op
        calls.append(call)
        extra_meta.append((M, N, K, r0, 3900, 7, 9, 11, 13, op))
    plan = fm.fm_plan_create(calls, P16, fm.FM_ALGO_LIMB_TC)
    plan.run()
    want = expected(orc, Cf, Af, Bf, meta + extra_meta)
    assert np.array_equal(MC.read(), want)
    plan.close()


@pytest.mark.parametrize("fused", [0, 1])
def test_limb_batched_graph_capture_and_replay(env, orc, fused):
    import torch
    fm, dev = env
    MC, MA, MB, Cf, Af, Bf, calls, meta = make_batch(fm, dev, 24, seed=11, lt=7)
    plan = fm.fm_plan_create(calls, P16, fm.FM_ALGO_LIMB_TC, fm.opts(fused_batch=fused))
    assert plan.launches == (1 if fused else 3)
    fm.fm_get_last_device_status()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(stream=s)
    torch.cuda.synchronize()
    assert np.array_equal(MC.read(), Cf)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(MC.read(), expected(orc, Cf, Af, Bf, meta, times=2))
    plan.close()


def test_limb_batched_rejects_pairs_and_overlap(env):
    fm, dev = env
    M = MortonMatrix(fm, dev, 1, 6)
    N = MortonMatrix(fm, dev, 1, 6)
    call = fm.fm_gemm_call()
    call.C, call.A, call.B = M.sub(0, 0, 8, 8), N.sub(8, 8, 8, 8), N.sub(4, 4, 8, 8)
    with pytest.raises(fm.FmError):
        fm.fm_plan_create([call], P16, fm.FM_ALGO_LIMB_TC, fm.opts(cta_pair=1))
    call.A = M.sub(4, 4, 8, 8)  # overlaps C
    with pytest.raises(fm.FmError):
        fm.fm_plan_create([call], P16, fm.FM_ALGO_LIMB_TC)


@pytest.mark.parametrize("lt,k_chunk,lo,hi,count,block,big,p", [
    (3, 0, 1, 40, 48, 64, 512, P16),          # T' = 8: a stage's 8-row runs of B cross tile rows
    (5, 64, 1, 300, 24, 320, 2048, P16),      # a fold of every product after every stage
    (6, 0, 300, 1100, 4, 1152, 4096, P16),    # K beyond 960: folds of the outer products as well
    (7, 128, 32, 600, 12, 640, 4096, 257),
])
def test_fused_batch_matches_oracle_and_plane_form(env, orc, lt, k_chunk, lo, hi, count, block, big, p):
    # the one-launch fused batch (operands split on the fly, K window and output
    # columns shifted by the operands' column offsets mod 4) against the oracle
    # and against the three-launch form with limb planes in a workspace
    fm, dev = env
    MC, MA, MB, Cf, Af, Bf, calls, meta = make_batch(fm, dev, count, seed=lt * 7 + k_chunk, lt=lt, lo=lo,
                                                     hi=hi, block=block, big=big)
    if p < P16:
        Cf, Af, Bf = Cf % p, Af % p, Bf % p
        MC.load(Cf)
        MA.load(Af)
        MB.load(Bf)
    if count >= 12:  # random column offsets: every shift of A and of B occurs
        assert {int(m[6]) % 4 for m in meta} == {0, 1, 2, 3} == {int(m[8]) % 4 for m in meta}
    plan = fm.fm_plan_create(calls, p, fm.FM_ALGO_LIMB_TC, fm.opts(k_chunk=k_chunk, fused_batch=1))
    assert plan.launches == 1
    saved = MC.t.clone()
    plan.run()
    got = MC.read()
    assert fm.fm_get_last_device_status() == 0
    assert np.array_equal(got, expected(orc, Cf, Af, Bf, meta, p=p))
    MC.t.copy_(saved)
    staged = fm.fm_plan_create(calls, p, fm.FM_ALGO_LIMB_TC, fm.opts(k_chunk=k_chunk))
    assert staged.launches == 3
    staged.run()
    assert np.array_equal(MC.read(), got)
    plan.close()
    staged.close()


def test_fused_batch_tiny_and_shifted_calls(env, orc):
    # every combination of A's and B's column offset mod 4 with M, N, K in 1..7
    fm, dev = env
    lt = 5
    Cf = fm_inputs.uniform_residues(41, (1024, 1024), P16, 1)
    Af = fm_inputs.uniform_residues(41, (1024, 1024), P16, 2)
    Bf = fm_inputs.uniform_residues(41, (1024, 1024), P16, 3)
    MC, MA, MB = (MortonMatrix(fm, dev, 5, lt, fill=x) for x in (Cf, Af, Bf))
    calls, meta = [], []
    dims = fm_inputs.integers(42, 3 * 64, 1, 7).reshape(64, 3)
    for c in range(64):
        M, N, K = (int(x) for x in dims[c])
        ra, rb = c % 4, (c // 4) % 4
        cr, cc = (c // 8) * 16, (c % 8) * 16 + (c // 16)
        ar, ac = 3 * c, 100 + 8 * c + ra
        br, bc = 5 * c, 200 + 8 * c + rb
        call = fm.fm_gemm_call()
        call.C, call.A, call.B = MC.sub(cr, cc, M, N), MA.sub(ar, ac, M, K), MB.sub(br, bc, K, N)
        call.op = c % 3
        calls.append(call)
        meta.append((M, N, K, cr, cc, ar, ac, br, bc, c % 3))
    plan = fm.fm_plan_create(calls, P16, fm.FM_ALGO_LIMB_TC, fm.opts(fused_batch=1))
    assert plan.launches == 1
    plan.run()
    assert fm.fm_get_last_device_status() == 0
    assert np.array_equal(MC.read(), expected(orc, Cf, Af, Bf, meta))
    plan.close()


def test_fused_batch_rejects_small_tiles_and_other_forms(env, orc):
    # T' = 4 operands (an 8-row run of B may cross two tile rows) and forms
    # other than two-limb Karatsuba are not fused; the plane form runs them
    fm, dev = env
    MC, MA, MB, Cf, Af, Bf, calls, meta = make_batch(fm, dev, 6, seed=5, lt=2, lo=8, hi=60, block=64, big=256)
    with pytest.raises(fm.FmError):
        fm.fm_plan_create(calls, P16, fm.FM_ALGO_LIMB_TC, fm.opts(fused_batch=1))
    for o in ({"no_karatsuba": 1}, {"block_n": 256}):
        with pytest.raises(fm.FmError):
            fm.fm_plan_create(calls[:1], P16, fm.FM_ALGO_LIMB_TC, fm.opts(fused_batch=1, **o))
    with pytest.raises(fm.FmError):
        fm.fm_plan_create(calls[:1], P31, fm.FM_ALGO_LIMB_TC, fm.opts(fused_batch=1))
    plan = fm.fm_plan_create(calls, P16, fm.FM_ALGO_LIMB_TC)
    assert plan.launches == 3
    plan.run()
    assert np.array_equal(MC.read(), expected(orc, Cf, Af, Bf, meta))
    plan.close()


def test_batch_workload_full_size_against_oracle(env, orc):
    # The bench's batch at full size and in the launch configuration it times:
    # 4096 calls C -= A*B mod 65521 with M, N, K uniform in [32, 512], each in
    # its own 512 x 512 cell of a 32768 x 32768 C, A and B random rectangles of
    # 16384 x 16384 matrices, T' = 64. C starts random inside every call's part.
    # The tensor-core limb plan (3 launches) is compared with the oracle call by
    # call, every entry; the fused limb plan and the decomposed plain plan must
    # give the same matrix.
    import torch
    fm, dev = env
    p, seed, count, hi, big, lt = P16, 5, 4096, 512, 16384, 6
    rows, cells = fm_inputs.batch_workload(seed, count, 32, hi, big)
    nC = cells * hi
    lgA = (big >> lt).bit_length() - 1
    lgC = (nC >> lt).bit_length() - 1
    Af = fm_inputs.uniform_residues(seed, (big, big), p, 1)
    Bf = fm_inputs.uniform_residues(seed, (big, big), p, 2)
    MA = MortonMatrix(fm, dev, lgA, lt, fill=Af)
    MB = MortonMatrix(fm, dev, lgA, lt, fill=Bf)
    Cf = np.zeros((nC, nC), dtype=np.uint32)
    for c in range(count):
        M, N, K, rC, cC = (int(x) for x in rows[c, :5])
        Cf[rC:rC + M, cC:cC + N] = fm_inputs.uniform_residues(seed, (M, N), p, 100 + c)
    MC = MortonMatrix(fm, dev, lgC, lt, fill=Cf)
    calls = []
    for c in range(count):
        M, N, K, rC, cC, rA, cA, rB, cB = (int(x) for x in rows[c])
        call = fm.fm_gemm_call()
        call.C, call.A, call.B = MC.sub(rC, cC, M, N), MA.sub(rA, cA, M, K), MB.sub(rB, cB, K, N)
        call.op = fm.FM_OP_SUB
        calls.append(call)
    saved = MC.t.clone()
    plan = fm.fm_plan_create(calls, p, fm.FM_ALGO_LIMB_TC)
    assert plan.launches == 3
    plan.run()
    got = MC.read()
    assert fm.fm_get_last_device_status() == 0
    for c in range(count):
        M, N, K, rC, cC, rA, cA, rB, cB = (int(x) for x in rows[c])
        want = orc.gemm_modp(Cf[rC:rC + M, cC:cC + N], Af[rA:rA + M, cA:cA + K], Bf[rB:rB + K, cB:cB + N], p,
                             fm.FM_OP_SUB)
        assert np.array_equal(got[rC:rC + M, cC:cC + N], want), c
        got[rC:rC + M, cC:cC + N] = Cf[rC:rC + M, cC:cC + N]
    assert np.array_equal(got, Cf)  # nothing outside the calls' parts changed
    del got
    limb = MC.t.clone()
    plan.close()
    for algo, o in ((fm.FM_ALGO_LIMB_TC, fm.opts(fused_batch=1)), (fm.FM_ALGO_PLAIN, None)):
        MC.t.copy_(saved)
        other = fm.fm_plan_create(calls, p, algo, o)
        other.run()
        torch.cuda.synchronize()
        assert fm.fm_get_last_device_status() == 0
        assert torch.equal(MC.t, limb), algo
        other.close()
    del MA, MB, MC, saved, limb
    torch.cuda.empty_cache()
