"""The measured pipe rates that serve as the non-tensor forms' rooflines."""
import pytest

from gpu_util import lib_and_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


def test_measured_rates_are_plausible(env):
    # 152 SMs at up to ~2.1 GHz: every scalar pipe is below 152 * 128 lanes *
    # 2.1e9 = 41 T multiply-adds/s and far above zero; the warp-level int8 MMA
    # is faster than any scalar pipe
    fm, _ = env
    r = {k: fm.fm_measure_peak(k, 1 << 12) / 1e12 for k in (
        fm.FM_PEAK_IMAD_WIDE, fm.FM_PEAK_IMAD32, fm.FM_PEAK_DFMA, fm.FM_PEAK_FFMA, fm.FM_PEAK_MMA_S8)}
    for k in (fm.FM_PEAK_IMAD_WIDE, fm.FM_PEAK_IMAD32, fm.FM_PEAK_FFMA):
        assert 1.0 < r[k] < 45.0, (k, r[k])
    assert 0.1 < r[fm.FM_PEAK_DFMA] < 45.0
    assert r[fm.FM_PEAK_MMA_S8] > r[fm.FM_PEAK_FFMA]
    assert fm.fm_get_last_device_status() == 0


def test_measure_peak_rejects_bad_arguments(env):
    fm, _ = env
    with pytest.raises(fm.FmError):
        fm.fm_measure_peak(9)
    with pytest.raises(fm.FmError):
        fm.fm_measure_peak(fm.FM_PEAK_DFMA, 0)
