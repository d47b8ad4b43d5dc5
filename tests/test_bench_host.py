"""Host-side logic of bench.py that needs no GPU: the clock sampler's decoding of
NVML clock-event reasons and its summary, through a fake NVML library."""
import ctypes
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class _FakeNvml:
    """Stands in for libnvidia-ml: fixed clocks and a given reason bit mask."""

    def __init__(self, sm, mx, bits):
        self.sm, self.mx, self.bits = sm, mx, bits

    def nvmlDeviceGetClockInfo(self, hd, kind, out):
        ctypes.cast(out, ctypes.POINTER(ctypes.c_uint)).contents.value = self.sm
        return 0

    def nvmlDeviceGetMaxClockInfo(self, hd, kind, out):
        ctypes.cast(out, ctypes.POINTER(ctypes.c_uint)).contents.value = self.mx
        return 0

    def reasons(self, hd, out):
        ctypes.cast(out, ctypes.POINTER(ctypes.c_ulonglong)).contents.value = self.bits
        return 0


def _sampler(sm, mx, bits):
    import bench
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.gpu, c.rows, c.source = 0, [], "nvml"
    fake = _FakeNvml(sm, mx, bits)
    c._nvml = (fake, None, fake.reasons)
    return c


def test_reason_bits_decode_to_the_throttle_names():
    # sw_power_cap 0x4, hw_slowdown 0x8, sw_thermal 0x20, hw_thermal 0x40 (NVML's bit values);
    # 0x1 (GPU idle) and 0x100 (display clock) are not throttle reasons the bench reports
    c = _sampler(1500, 2032, 0x4 | 0x40 | 0x1 | 0x100)
    c._sample_nvml()
    s = c.summary()
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["sm_mhz"] == 1500.0 and s["sm_max_mhz"] == 2032.0 and s["samples"] == 1


def test_summary_is_the_median_and_the_union_of_reasons():
    c = _sampler(2032, 2032, 0)
    for sm, bits in ((2032, 0), (1900, 0x8), (2000, 0), (1100, 0x20), (2032, 0)):
        c._nvml[0].sm, c._nvml[0].bits = sm, bits
        c._sample_nvml()
    s = c.summary()
    assert s["sm_mhz"] == 2000.0
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert s["samples"] == 5 and s["source"] == "nvml"


def test_no_samples_reports_none():
    c = _sampler(2032, 2032, 0)
    s = c.summary()
    assert s["sm_mhz"] is None and s["sm_max_mhz"] is None and s["reasons"] == [] and s["samples"] == 0


def test_sampler_runs_and_stops_without_a_gpu():
    # on a machine without the NVML library the sampler falls back to nvidia-smi; either way
    # entering and leaving it must not raise or hang
    import bench
    c = bench.ClockSampler(0)
    assert c.source in ("nvml", "nvidia-smi")
    with c:
        pass
    assert isinstance(c.summary()["samples"], int)
