"""cvo_measure_throughput: the FP32 FMA and ex2 rates that the benchmark
takes as its roofline denominators are measured, not counted, so they must
lie between a fraction of the unit-count ceiling and that ceiling at any
clock the part can run at (an FMA counts 2 FLOPs; 128 FP32 lanes per SM)."""
import pytest

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu

MAX_CLOCK_HZ = 2.2e9   # above the part's highest SM clock
MIN_CLOCK_HZ = 0.5e9


def test_measured_rates_within_the_units_ceiling():
    t = cvo.cvo_measure_throughput()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert t["sms"] == sms
    assert sms * 128 * 2 * MIN_CLOCK_HZ <= t["ffma_flops"] <= sms * 128 * 2 * MAX_CLOCK_HZ
    # the ex2 unit: at least 4 and at most 64 evaluations per SM per clock
    assert sms * 4 * MIN_CLOCK_HZ <= t["ex2_per_s"] <= sms * 64 * MAX_CLOCK_HZ
    assert t["ms_ffma"] > 0.0 and t["ms_ex2"] > 0.0


def test_null_output_rejected():
    import ctypes
    lib = cvo.load_library()
    assert lib.cvo_measure_throughput(None, None) == int(cvo.Status.ERR_INVALID_ARG)
    assert "NULL" in cvo.cvo_last_error()
