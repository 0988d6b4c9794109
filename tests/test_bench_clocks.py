"""bench.py's clock record: the NVML reader decodes clocks and event reasons (a fake
NVML stands in for the library; the reader only queries)."""
import ctypes
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class FakeNvml:
    def __init__(self, reasons):
        self.r = reasons
        self.calls = 0

    def nvmlDeviceGetClockInfo(self, h, kind, ref):
        assert kind == 1  # the SM clock
        self.calls += 1
        ref._obj.value = 1965 if self.calls % 2 else 2070
        return 0

    def nvmlDeviceGetMaxClockInfo(self, h, kind, ref):
        ref._obj.value = 2070
        return 0

    def nvmlDeviceGetCurrentClocksEventReasons(self, h, ref):
        ref._obj.value = self.r
        return 0


def sampler(reasons):
    s = bench.NvmlClockSampler.__new__(bench.NvmlClockSampler)
    s.ct, s.nvml, s.h, s.period = ctypes, FakeNvml(reasons), None, 0.001
    s.get_reasons = s.nvml.nvmlDeviceGetCurrentClocksEventReasons
    s.samples, s.reasons, s.stop_flag = [], 0, False
    return s


def test_reasons_and_median():
    s = sampler(0x1 | 0x4)  # idle + software power cap
    s.start()
    time.sleep(0.05)
    d = s.stop()
    assert d["samples"] >= 5 and d["sm_max_mhz"] == 2070
    assert d["sm_mhz"] in (1965, 2070, (1965 + 2070) / 2)
    assert d["reasons"] == ["sw_power_cap"]


def test_slowdowns_are_named():
    s = sampler(0x8 | 0x20 | 0x40)
    s.start()
    time.sleep(0.02)
    assert s.stop()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_fallback_without_nvml():
    # without a GPU driver the factory falls back to the nvidia-smi reader
    s = bench.clock_sampler(0)
    assert isinstance(s, (bench.NvmlClockSampler, bench.ClockSampler))
