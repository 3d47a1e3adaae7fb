"""Host logic of bench.py that needs no GPU: the clock-sample summary (median SM clock, throttle reasons), the
roofline denominators (the measured copy rate, else the fallback), and the DRAM-traffic records, which count
only while the kernel source they were taken from is unchanged."""
import importlib.util
import json
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_summarize_clocks(bench):
    lines = [
        "0, 2070, 2070, 990.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1001.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 995.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "not a sample",
        "0, [N/A], 2070, 1.0, 0x0, Active, Active, Active, Active",  # no clock reading: skipped whole
    ]
    assert bench.summarize_clocks(lines) == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                                             "samples": 3}
    assert bench.summarize_clocks([]) is None
    assert bench.summarize_clocks(["garbage", ""]) is None
    hot = bench.summarize_clocks(["0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active",
                                  "0, 1600, 2070, 1400, 0x8, Not Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert hot["sm_mhz"] == 1550.0 and hot["samples"] == 2


def test_peaks_measured_or_fallback(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7012.5, "bf16_tflops": 1900.0}))
    assert bench.peaks() == (7012.5, "measured")
    (tmp_path / "MEASURED_PEAKS.json").write_text("{not json")
    assert bench.peaks() == (6800.0, "fallback")


@pytest.mark.parametrize("which", ["fp64", "ff", "oz"])
def test_traffic_record_counts_only_for_its_kernel_source(bench, tmp_path, monkeypatch, which):
    src, rec = bench.AX_SOURCES[which]
    with open(os.path.join(ROOT, "profiles", rec)) as fh:
        t = json.load(fh)
    nx = int(t["nx"])
    per_elem = float(t["dram_bytes_per_element"])
    # the record is self-consistent: bytes per element = (read + write) / captured elements
    assert per_elem == pytest.approx((t["dram_bytes_read"] + t["dram_bytes_write"]) / t["captured_elements"],
                                     rel=1e-4)
    # it scales with the elements of the launch while its source hash matches; otherwise, and at another nx,
    # there is no traffic figure
    expect = per_elem * 32768 if t["source_sha"] == bench.kernel_source_sha(which) else None
    assert bench.traffic_from_profile(nx, 32768, which) == (pytest.approx(expect) if expect else None)
    assert bench.traffic_from_profile(nx + 1, 32768, which) is None
    # a changed kernel source voids the record
    csrc = tmp_path / "paper_2011_04981_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copytree(os.path.join(ROOT, "profiles"), tmp_path / "profiles")
    with open(os.path.join(ROOT, "paper_2011_04981_gb300", "csrc", src), "rb") as fh:
        body = fh.read()
    (csrc / src).write_bytes(body + b"\n// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_source_sha(which) != t["source_sha"]
    assert bench.traffic_from_profile(nx, 32768, which) is None
    # an unchanged copy of the source keeps it
    (csrc / src).write_bytes(body)
    if expect:
        assert bench.traffic_from_profile(nx, 32768, which) == pytest.approx(expect)
