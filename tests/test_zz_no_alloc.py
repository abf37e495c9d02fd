"""fm_gemm_modp_noalloc: the tensor-core limb product with no device allocation.

Some callers cannot let the library call cudaMalloc: programs whose device
memory comes only from their own allocator or a fixed budget (a serving process
that reserves the GPU's memory for its pool at start-up), and code that must not
stall on the device synchronisation cudaMalloc implies. For them the library
keeps the limb planes in a fixed 64 MiB device array instead of allocated
workspace. These checks call that entry point through the C ABI on two calls in
a row -- the second one reuses the array the first one left behind -- and
compare each result with the CPU oracle, entry by entry, and with the existing
entry point, fm_gemm_modp's limb form, bit for bit. They also check that a call
leaves the device's free memory and torch's allocator as they were, that K = 0
calls touch only what they should, that a device-side wait that runs out on
this path reaches fm_get_last_device_status, and that a product needing more
than the fixed scratch is refused.

Kept in a file of its own that pytest collects last; the checks pass in a fresh
process and after the other tests alike.
"""
import time

import numpy as np
import pytest

import fm_inputs
from gpu_util import MortonMatrix, grid_for, lib_and_device

pytestmark = pytest.mark.gpu

P16, P31 = 65521, 2147483647


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def _problem(env, p, M, N, K, offs, lts, seed):
    """Random Morton-hybrid C, A, B holding the sub-matrices at offs; returns
    the device matrices and the host arrays they were filled from."""
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
    mats = tuple(MortonMatrix(fm, dev, lg, lt, fill=x) for lg, lt, x in
                 ((lgC, ltC, Cf), (lgA, ltA, Af), (lgB, ltB, Bf)))
    return {"p": p, "M": M, "N": N, "K": K, "offs": offs, "mats": mats, "host": (Cf, Af, Bf)}


def _subs(pb, C=None):
    MC, MA, MB = pb["mats"]
    rC, cC, rA, cA, rB, cB = pb["offs"]
    M, N, K = pb["M"], pb["N"], pb["K"]
    return (C or MC).sub(rC, cC, M, N), MA.sub(rA, cA, M, K), MB.sub(rB, cB, K, N)


def _oracle(orc, pb, op):
    Cf, Af, Bf = pb["host"]
    rC, cC, rA, cA, rB, cB = pb["offs"]
    M, N, K = pb["M"], pb["N"], pb["K"]
    want = Cf.copy()
    want[rC:rC + M, cC:cC + N] = orc.gemm_modp(Cf[rC:rC + M, cC:cC + N], Af[rA:rA + M, cA:cA + K],
                                               Bf[rB:rB + K, cB:cB + N], pb["p"], op)
    return want


def test_noalloc_matches_oracle_and_existing_entry_on_two_calls(env, orc):
    fm, dev = env
    # first call: p = 65521 (residue folded into the accumulator), ragged and
    # misaligned sub-matrices, mixed T'
    first = _problem(env, P16, 700, 900, 1500, (13, 70, 5, 33, 100, 3), (7, 6, 5), seed=21)
    # second call right after: a different modulus, shape and limb count, so the
    # shared scratch holds the first call's planes when it starts
    second = _problem(env, P31, 513, 300, 1100, (0, 5, 7, 0, 3, 9), (6, 7, 6), seed=22)
    todo = ((first, fm.FM_OP_SUB), (second, fm.FM_OP_ADD))
    got = []
    for pb, op in todo:
        fm.fm_gemm_modp_noalloc(*_subs(pb), pb["p"], op)
        got.append(pb["mats"][0].read())
    assert fm.fm_get_last_device_status() == 0
    for (pb, op), g in zip(todo, got):
        assert np.array_equal(g, _oracle(orc, pb, op)), pb["p"]
    # the existing entry point on fresh copies of the same C gives the same integers
    for (pb, op), g in zip(todo, got):
        MC = pb["mats"][0]
        ref = MortonMatrix(fm, dev, MC.lg, MC.lt, fill=pb["host"][0])
        fm.fm_gemm_modp(*_subs(pb, C=ref), pb["p"], op, fm.FM_ALGO_LIMB_TC)
        assert np.array_equal(ref.read(), g), pb["p"]


def test_noalloc_leaves_device_memory_as_it_was(env, orc):
    # after one call of a shape (which loads the kernels it needs), a second
    # call of that shape changes neither the device's free memory nor what
    # torch's allocator holds
    import torch
    fm, dev = env
    pb = _problem(env, P16, 600, 520, 1300, (3, 0, 0, 9, 17, 4), (6, 6, 7), seed=24)
    subs = _subs(pb)
    fm.fm_gemm_modp_noalloc(*subs, P16, fm.FM_OP_SUB)
    torch.cuda.synchronize()
    free0, alloc0, reserved0 = torch.cuda.mem_get_info(dev)[0], torch.cuda.memory_allocated(dev), \
        torch.cuda.memory_reserved(dev)
    fm.fm_gemm_modp_noalloc(*subs, P16, fm.FM_OP_SUB)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    assert torch.cuda.memory_allocated(dev) == alloc0 and torch.cuda.memory_reserved(dev) == reserved0
    # and the two calls subtracted the product twice
    Cf, Af, Bf = pb["host"]
    rC, cC, rA, cA, rB, cB = pb["offs"]
    M, N, K = pb["M"], pb["N"], pb["K"]
    want = Cf.copy()
    blk = Cf[rC:rC + M, cC:cC + N]
    for _ in range(2):
        blk = orc.gemm_modp(blk, Af[rA:rA + M, cA:cA + K], Bf[rB:rB + K, cB:cB + N], P16, fm.FM_OP_SUB)
    want[rC:rC + M, cC:cC + N] = blk
    assert np.array_equal(pb["mats"][0].read(), want)
    assert fm.fm_get_last_device_status() == 0


def test_noalloc_k0_calls(env):
    # K = 0: FM_OP_SET zeroes exactly the C sub-matrix, ADD and SUB leave C as is
    fm, dev = env
    pb = _problem(env, P16, 70, 90, 0, (5, 3, 1, 0, 0, 2), (5, 6, 6), seed=25)
    MC = pb["mats"][0]
    Cf = pb["host"][0]
    for op in (fm.FM_OP_ADD, fm.FM_OP_SUB):
        fm.fm_gemm_modp_noalloc(*_subs(pb), P16, op)
        assert np.array_equal(MC.read(), Cf)
    fm.fm_gemm_modp_noalloc(*_subs(pb), P16, fm.FM_OP_SET)
    want = Cf.copy()
    want[5:75, 3:93] = 0
    assert np.array_equal(MC.read(), want)
    assert fm.fm_get_last_device_status() == 0


def test_noalloc_expired_wait_reaches_status(env, orc):
    # A wait that runs out on this path raises FM_ETIMEOUT in the fixed
    # scratch's own status word; fm_get_last_device_status reports it once and
    # clears it, and the next call computes normally. The test hook runs the
    # library's bounded mbarrier wait on a phase nothing completes (2 s limit).
    import torch
    fm, dev = env
    assert fm.fm_get_last_device_status() == 0
    t0 = time.perf_counter()
    fm.fm_debug_expire_wait(2)
    torch.cuda.synchronize()
    assert 1.5 < time.perf_counter() - t0 < 30.0
    assert fm.fm_get_last_device_status() == fm.FM_ETIMEOUT
    assert fm.fm_get_last_device_status() == 0
    pb = _problem(env, P16, 200, 130, 300, (1, 2, 3, 4, 5, 6), (6, 6, 6), seed=26)
    fm.fm_gemm_modp_noalloc(*_subs(pb), P16, fm.FM_OP_SUB)
    assert np.array_equal(pb["mats"][0].read(), _oracle(orc, pb, fm.FM_OP_SUB))
    assert fm.fm_get_last_device_status() == 0


def test_noalloc_refuses_products_beyond_its_scratch(env):
    fm, dev = env
    pb = _problem(env, P16, 4096, 4096, 4096, (0, 0, 0, 0, 0, 0), (7, 7, 7), seed=23)
    MC = pb["mats"][0]
    before = MC.read()
    with pytest.raises(fm.FmError) as err:
        fm.fm_gemm_modp_noalloc(*_subs(pb), P16, fm.FM_OP_SUB)
    assert err.value.code == fm.FM_ETOOBIG
    assert np.array_equal(MC.read(), before)
