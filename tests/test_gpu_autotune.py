"""The autotuner: measured choice of form and options, then FM_ALGO_AUTO uses it
and stays bit-exact against the oracle."""
import numpy as np
import pytest

from gpu_util import lib_and_device
from test_gpu_gemm import run_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


@pytest.mark.parametrize("p", [65521, 2147483647])
def test_autotune_then_auto_is_exact(env, orc, p):
    fm = env[0]
    fm.fm_autotune_clear()
    M, N, K = 300, 520, 1000
    r = fm.fm_autotune(M, N, K, p)
    assert r.algo in (fm.FM_ALGO_PLAIN, fm.FM_ALGO_LIMB_TC)
    assert r.candidates >= 2 and r.ms > 0 and r.gops > 0
    hit = fm.fm_autotune_lookup(M, N, K, p)
    assert hit is not None and hit.algo == r.algo
    for lts in ((6, 6, 6), (7, 5, 6)):
        got, want = run_case(env, orc, p, 2, fm.FM_ALGO_AUTO, M, N, K, (3, 5, 0, 9, 7, 0), lts, seed=11)
        assert np.array_equal(got, want)
    fm.fm_autotune_clear()


def test_autotune_flags(env):
    fm = env[0]
    r = fm.fm_autotune(256, 256, 256, 65521, fm.FM_TUNE_NO_LIMB)
    assert r.algo == fm.FM_ALGO_PLAIN and r.log2_T in (5, 6)
    r = fm.fm_autotune(256, 256, 256, 65521, fm.FM_TUNE_NO_PLAIN)
    assert r.algo == fm.FM_ALGO_LIMB_TC
    with pytest.raises(fm.FmError):
        fm.fm_autotune(256, 256, 256, 65521, fm.FM_TUNE_NO_PLAIN | fm.FM_TUNE_NO_LIMB)
    fm.fm_autotune_clear()


@pytest.mark.parametrize("p,lt", [(65521, 6), (65521, 7), (2147483647, 5)])
def test_autotune_batch_then_auto_plan_is_exact(env, orc, p, lt):
    # the batch tuner times the plan forms on the batch itself without changing
    # C; an FM_ALGO_AUTO plan of that batch then takes the remembered form and
    # matches the oracle
    from test_gpu_batched import expected, make_batch
    fm = env[0]
    fm.fm_autotune_clear()
    MC, MA, MB, Cf, Af, Bf, calls, meta = make_batch(fm, env[1], 40, seed=lt + 1, lt=lt)
    # (residues below 65521 are residues mod 2^31 - 1 as well)
    r = fm.fm_autotune_batch(calls, p)
    assert r.algo in (fm.FM_ALGO_PLAIN, fm.FM_ALGO_LIMB_TC) and r.ms > 0 and r.gops > 0
    assert r.candidates >= 2 and r.log2_T == lt
    if lt == 7:
        assert r.algo == fm.FM_ALGO_LIMB_TC  # the decomposed forms take T' = 32 or 64 only
    assert np.array_equal(MC.read(), Cf)  # tuning ran on scratch copies of C
    plan = fm.fm_plan_create(calls, p, fm.FM_ALGO_AUTO)
    if r.algo == fm.FM_ALGO_LIMB_TC:
        assert plan.launches == (1 if r.opts.fused_batch else 3)
    else:
        assert plan.launches == 1
    plan.run()
    assert fm.fm_get_last_device_status() == 0
    assert np.array_equal(MC.read(), expected(orc, Cf, Af, Bf, meta, p=p))
    plan.close()
    fm.fm_autotune_clear()
