"""Failure detection without a GPU fault: bounded device waits expire into
FM_ETIMEOUT and leave the context usable; FM_TRACE records calls."""
import os
import time

import numpy as np
import pytest

import fm_inputs
from gpu_util import MortonMatrix, grid_for, lib_and_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def small_product_ok(fm, dev, orc):
    p = 65521
    A = fm_inputs.uniform_residues(3, (100, 70), p, 1)
    B = fm_inputs.uniform_residues(3, (70, 90), p, 2)
    lt = 6
    MA = MortonMatrix(fm, dev, grid_for(100, 70, lt), lt, fill=A)
    MB = MortonMatrix(fm, dev, grid_for(70, 90, lt), lt, fill=B)
    MC = MortonMatrix(fm, dev, grid_for(100, 90, lt), lt)
    fm.fm_gemm_modp(MC.sub(0, 0, 100, 90), MA.sub(0, 0, 100, 70), MB.sub(0, 0, 70, 90), p, 0,
                    fm.FM_ALGO_LIMB_TC)
    assert fm.fm_get_last_device_status() == 0
    return np.array_equal(MC.read(100, 90), orc.gemm_modp(None, A, B, p, 0))


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_expires_into_status(env, orc, which):
    # which 0: an mbarrier phase nothing completes; 1: a grid barrier one CTA
    # never reaches. The wait gives up after 2 s, the kernel exits, the status
    # word says FM_ETIMEOUT, and the next product runs normally.
    import torch
    fm, dev = env
    assert fm.fm_get_last_device_status() == 0
    t0 = time.perf_counter()
    fm.fm_debug_expire_wait(which)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert 1.5 < waited < 30.0
    assert fm.fm_get_last_device_status() == fm.FM_ETIMEOUT
    assert fm.fm_get_last_device_status() == 0  # reading clears it
    assert small_product_ok(fm, dev, orc)


def test_debug_hook_rejects_unknown_kind(env):
    fm, _ = env
    with pytest.raises(fm.FmError):
        fm.fm_debug_expire_wait(7)


def test_trace_lines(env, orc, tmp_path):
    fm, dev = env
    log = tmp_path / "trace.txt"
    os.environ["FM_TRACE"] = str(log)
    try:
        assert small_product_ok(fm, dev, orc)
    finally:
        del os.environ["FM_TRACE"]
    text = log.read_text()
    assert "gemm_modp limb M=100 N=90 K=70 p=65521" in text and "tiles=" in text
    assert small_product_ok(fm, dev, orc)
    assert log.read_text() == text  # tracing is off again
