"""fm_gemm_modp_noalloc: the tensor-core limb product with no device allocation.

Some callers cannot let the library call cudaMalloc: code that runs while a
CUDA graph is being captured, and programs whose device memory comes only from
their own allocator or a fixed budget. For them the library keeps the limb
planes in a fixed 64 MiB device array instead of allocated workspace. These
checks call that entry point through the C ABI and compare it with
fm_gemm_modp's limb form (the existing entry point) bit for bit, on two calls
in a row -- the second one reuses the array the first one left behind -- and
check that a product needing more than the fixed scratch is refused.

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import fm_inputs
from gpu_util import MortonMatrix, grid_for, lib_and_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def _problem(env, p, M, N, K, offs, lts, seed):
    fm, dev = env
    rC, cC, rA, cA, rB, cB = offs
    ltC, ltA, ltB = lts
    lgC = grid_for(rC + M, cC + N, ltC)
    lgA = grid_for(rA + M, cA + K, ltA)
    lgB = grid_for(rB + K, cB + N, ltB)
    nC, nA, nB = (1 << lgC) << ltC, (1 << lgA) << ltA, (1 << lgB) << ltB
    MC = MortonMatrix(fm, dev, lgC, ltC, fill=fm_inputs.uniform_residues(seed, (nC, nC), p, 1))
    MA = MortonMatrix(fm, dev, lgA, ltA, fill=fm_inputs.uniform_residues(seed, (nA, nA), p, 2))
    MB = MortonMatrix(fm, dev, lgB, ltB, fill=fm_inputs.uniform_residues(seed, (nB, nB), p, 3))
    # MA and MB travel with the problem: the fm_sub structs hold raw pointers
    return MC, MA.sub(rA, cA, M, K), MB.sub(rB, cB, K, N), (rC, cC, M, N), (MA, MB)


def _both(env, p, op, problem):
    """Runs the no-allocation entry point on C and fm_gemm_modp's limb form on
    a copy of C; returns both full matrices."""
    fm, dev = env
    MC, sA, sB, (rC, cC, M, N), _ = problem
    ref = MortonMatrix(fm, dev, MC.lg, MC.lt)
    ref.t.copy_(MC.t)
    fm.fm_gemm_modp(ref.sub(rC, cC, M, N), sA, sB, p, op, fm.FM_ALGO_LIMB_TC)
    fm.fm_gemm_modp_noalloc(MC.sub(rC, cC, M, N), sA, sB, p, op)
    return MC.read(), ref.read()


def test_noalloc_matches_existing_entry_on_two_calls(env):
    fm, _ = env
    # first call: p = 65521 (residue folded into the accumulator), ragged and
    # misaligned sub-matrices, mixed T'
    first = _problem(env, 65521, 700, 900, 1500, (13, 70, 5, 33, 100, 3), (7, 6, 5), seed=21)
    got, want = _both(env, 65521, fm.FM_OP_SUB, first)
    assert np.array_equal(got, want)
    # second call right after: a different modulus, shape and limb count, so the
    # shared scratch holds the first call's planes when it starts
    second = _problem(env, 2147483647, 513, 300, 1100, (0, 5, 7, 0, 3, 9), (6, 7, 6), seed=22)
    got, want = _both(env, 2147483647, fm.FM_OP_ADD, second)
    assert np.array_equal(got, want)


def test_noalloc_refuses_products_beyond_its_scratch(env):
    fm, dev = env
    MC, sA, sB, (rC, cC, M, N), keep = _problem(env, 65521, 4096, 4096, 4096, (0, 0, 0, 0, 0, 0),
                                                (7, 7, 7), seed=23)
    before = MC.read()
    with pytest.raises(fm.FmError) as err:
        fm.fm_gemm_modp_noalloc(MC.sub(rC, cC, M, N), sA, sB, 65521, fm.FM_OP_SUB)
    assert err.value.code == fm.FM_ETOOBIG
    assert np.array_equal(MC.read(), before)
