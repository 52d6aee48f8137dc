"""Host logic of the bench's clock record: decoding NVML clock-event reasons and the summary
the JSON line carries (no GPU, no NVML: the sampler is built without its library)."""
import bench


def _sampler(samples, max_mhz=2070.0):
    s = bench.NvmlSampler.__new__(bench.NvmlSampler)
    s.samples = list(samples)
    s.max_mhz = max_mhz
    return s


def test_median_clock_and_no_reasons():
    out = _sampler([(2070.0, 0), (2055.0, 0), (2070.0, 0x1)]).summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [] and out["samples"] == 3 and out["source"] == "nvml"


def test_reason_bits_are_named():
    out = _sampler([(1980.0, 0x4), (1900.0, 0x8 | 0x40), (2000.0, 0x20)]).summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1980.0


def test_no_samples():
    out = _sampler([]).summary()
    assert out["sm_mhz"] is None and out["samples"] == 0
