"""Host logic of bench.py (no GPU, no NVML): the clock record (NVML clock-event reasons and the
summary the JSON line carries; the sampler is built without its library) and the source digest
that decides whether the profiled DRAM traffic still describes the compression kernels."""
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


def test_sources_digest_ignores_comments_but_not_code(tmp_path):
    import os
    import shutil
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = os.path.join(here, "paper_2511_04140_gb300", "csrc")
    dst = tmp_path / "paper_2511_04140_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in ("compress.cu", "falcon_device.cuh", "falcon_internal.h", "falcon_tables.h"):
        shutil.copy(os.path.join(src, f), dst / f)
    base = bench.compress_sources_digest(str(tmp_path))
    assert base == bench.compress_sources_digest(here)
    cu = dst / "compress.cu"
    text = cu.read_text()
    cu.write_text("// a new comment line\n/* and a block\n   comment */\n" + text.replace("\n", "\n\n", 3))
    assert bench.compress_sources_digest(str(tmp_path)) == base
    cu.write_text(text.replace("constexpr int kMetaShift = 47;", "constexpr int kMetaShift = 46;"))
    assert bench.compress_sources_digest(str(tmp_path)) != base


def test_failed_checks_finds_every_false_exactness_key():
    line = {"bit_exact": True, "batched": {"bit_exact": False, "oracle_equal": True},
            "serve": {"loads": [{"server": {"bit_exact": True}}, {"one": {"oracle_equal": False}}]}}
    assert bench.failed_checks(line) == ["line.batched.bit_exact", "line.serve.loads[1].one.oracle_equal"]
    assert bench.failed_checks({"bit_exact": True, "pipeline": {"bit_exact": True}}) == []
