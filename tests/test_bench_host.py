"""Host logic of bench.py that needs no GPU: the algorithmic FLOP count per
pair, the per-launch figures taken from the committed ncu summary (only
while its source hash matches the kernel source), and the parsing of the
clock samples (median SM clock, the throttle reasons seen)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

CSRC = os.path.join(ROOT, "paper_2012_03683_gb300", "csrc")
SWEEP_SRC = [os.path.join(CSRC, "cvo_sweep.cu"), os.path.join(CSRC, "cvo_sweep_dev.cuh")]


def test_grad_flops_per_pair():
    # offset 3, distance 5, scale 1, weight 1, accumulators 8; SE block 6d + 1; dot block 4d
    assert bench.grad_flops_per_pair([]) == 18
    assert bench.grad_flops_per_pair([("se", 3, 0.2, 1.0)]) == 18 + 19
    assert bench.grad_flops_per_pair([("se", 3, 0.2, 1.0), ("dot", 19, 1.0, 1.0)]) == 18 + 19 + 76


def test_cpu_sample_is_seeded_and_in_range():
    a = bench.sample_pairs(64)
    assert a == bench.sample_pairs(64) and len(a) == bench.CPU_SAMPLE_PAIRS == len(set(a))
    assert all(0 <= k < 64 for k in a)


def test_roofline_arithmetic():
    peaks = {"sm_max_mhz": 2000.0}
    r = bench.sweep_roofline("k", pairs_evaluated=1e9, sweep_ms_total=100.0, launches=50, fpp=76, peaks=peaks,
                             peak_src="measured", sms=152)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2e9 / 1e12)
    assert r["achieved"] == pytest.approx(1e9 * 76 / 0.1 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["sweep_ms_avg"] == pytest.approx(2.0) and r["pairs_per_launch"] == pytest.approx(2e7)
    assert r["sfu"]["achieved_ex2_per_s"] == pytest.approx(1e10)
    assert "unit counts" in r["peak_source"]


def test_roofline_against_measured_rates():
    """With the FP32 FMA and ex2 rates measured in the run, those are the
    denominators, and the unit count is reported beside them."""
    peaks = {"sm_max_mhz": 2000.0, "ffma_flops": 75e12, "ex2_per_s": 9e12}
    r = bench.sweep_roofline("k", pairs_evaluated=1e9, sweep_ms_total=100.0, launches=50, fpp=76, peaks=peaks,
                             peak_src="measured", sms=152)
    assert r["peak"] == pytest.approx(75.0)
    assert r["peak_unit_count"] == pytest.approx(152 * 128 * 2 * 2e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 75.0)
    assert r["sfu"]["peak_ex2_per_s"] == pytest.approx(9e12)
    assert r["peak_source"].startswith("of measured") and "of measured" in r["sfu"]["peak_source"]


def test_measured_rates_fall_back_to_unit_counts():
    class Fails:
        @staticmethod
        def cvo_measure_throughput():
            raise RuntimeError("no device")

    class Works:
        @staticmethod
        def cvo_measure_throughput():
            return {"ffma_flops": 7e13, "ex2_per_s": 1e13, "ms_ffma": 1.0, "ms_ex2": 1.0, "sms": 152}

    base = {"sm_max_mhz": 2070.0}
    assert bench.with_measured_throughput(Fails, base) == base
    got = bench.with_measured_throughput(Works, base)
    assert got["ffma_flops"] == 7e13 and got["ex2_per_s"] == 1e13 and "ffma_flops" not in base


def test_flops_per_pair():
    # offset 3, distance 5, scale 1, moments 19; SE block 3d + 1; dot block 2d
    assert bench.flops_per_pair([]) == 28
    assert bench.flops_per_pair([("se", 3, 0.2, 1.0)]) == 28 + 10
    assert bench.flops_per_pair([("se", 3, 0.2, 1.0), ("dot", 19, 1.0, 1.0)]) == 76


def test_profile_values_follow_the_source_hash(tmp_path):
    import hashlib
    import re
    text = open(os.path.join(ROOT, "profiles", "sweep_street-20k.md")).read()
    recorded = re.search(r"source_sha256:\s*([0-9a-f]{64})", text).group(1)
    current = hashlib.sha256(b"".join(open(f, "rb").read() for f in SWEEP_SRC)).hexdigest()
    traffic = bench.profile_value(SWEEP_SRC, "traffic_bytes_per_launch", "sweep_street-20k.md")
    winst = bench.profile_value(SWEEP_SRC, "warp_instructions_per_launch", "sweep_street-20k.md")
    if current == recorded:   # the summary was taken on this source: its figures are reported
        assert traffic is not None and 1e6 < traffic < 1e8
        assert winst is not None and 1e6 < winst < 1e9
    else:                     # the kernel changed since: none are
        assert traffic is None and winst is None
    # any other source (a changed kernel) gets no figure
    other = tmp_path / "changed.cu"
    other.write_text(open(SWEEP_SRC[0]).read() + "\n// changed\n")
    assert bench.profile_value([str(other), SWEEP_SRC[1]], "traffic_bytes_per_launch", "sweep_street-20k.md") is None
    assert bench.profile_value(SWEEP_SRC, "no_such_key", "sweep_street-20k.md") is None
    assert bench.profile_value(SWEEP_SRC, "traffic_bytes_per_launch", "no_such_profile.md") is None


class _FakeProc:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""

    def kill(self):
        pass


def test_clock_samples_parsed():
    rows = [
        "2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    s = bench.ClockSampler(0)
    s.proc = _FakeProc("\n".join(rows) + "\n")
    out = s.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == pytest.approx(2070.0)
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop() is None


def test_clock_sampler_end_to_end_with_a_stand_in_command(tmp_path):
    """start() waits for the first sample and stop() keeps it: a stand-in for
    nvidia-smi prints one sample line every 20 ms until it is terminated."""
    import subprocess
    import time
    script = tmp_path / "fake_smi.py"
    script.write_text(
        "import sys, time\n"
        "i = 0\n"
        "while True:\n"
        "    print(f'{2000 + i % 3}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active', flush=True)\n"
        "    i += 1\n"
        "    time.sleep(0.02)\n")
    s = bench.ClockSampler(0, command=[sys.executable, str(script)])
    s.start()
    assert s.first.startswith("20")
    time.sleep(0.15)
    out = s.stop()
    assert out["samples"] >= 3 and out["sm_max_mhz"] == 2070.0 and out["reasons"] == []
    assert 2000.0 <= out["sm_mhz"] <= 2002.0
    assert s.proc.poll() is not None   # the sampler process is gone


def test_clock_sampler_with_a_missing_command():
    s = bench.ClockSampler(0, command=["/nonexistent/nvidia-smi-stand-in"])
    s.start()
    assert s.proc is None and s.stop() is None
