"""Host logic of bench.py: the clock record (nvidia-smi rows are summarised over the samples taken inside the
timed region, one sampling interval of slack, throttle reasons are collected from those rows, and rows outside
the region are used only when none falls inside) and the key of the recorded DRAM traffic figure."""
import datetime
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def row(t, sm, reasons=("Not Active",) * 4):
    ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([ts, "0", str(sm), "2070", "900.5", "0x0", *reasons])


def test_samples_inside_the_region_decide_the_summary():
    t0 = 1.9e9
    lines = [row(t0 - 1.0, 500), row(t0 + 0.1, 2070), row(t0 + 0.3, 2055),
             row(t0 + 0.5, 2070, ("Not Active", "Not Active", "Not Active", "Active")), row(t0 + 2.0, 300)]
    s = bench.summarize_clocks(lines, t0, t0 + 0.45, 0.2)
    assert s["samples"] == 5 and s["samples_in_timed_region"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_all_rows_when_none_falls_inside_and_bad_rows_skipped():
    t0 = 1.9e9
    lines = ["garbage", row(t0 - 5.0, 1800), row(t0 + 5.0, 2000),
             ", ".join(["not a time", "0", "1900", "2070", "1", "0x0", "Active", "Not Active", "Not Active",
                        "Not Active"])]
    s = bench.summarize_clocks(lines, t0, t0 + 0.05, 0.2)
    assert s["samples"] == 3 and s["samples_in_timed_region"] == 0
    assert s["sm_mhz"] == 1900.0
    assert s["reasons"] == ["hw_slowdown"]
    assert bench.summarize_clocks([], t0, t0) is None


def test_traffic_figure_is_keyed_to_the_kernel_source(tmp_path, monkeypatch):
    """bench.py reports the recorded DRAM bytes per update only for the kernel source they were taken on."""
    import hashlib
    src = tmp_path / "kernels.cu"
    src.write_text("// kernel source\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(src))
    monkeypatch.setattr(bench, "SWEEP_FP32_TRAFFIC", {"kernel_source_sha256": h, "dram_bytes_per_update": 8.5})
    assert bench.traffic_per_update() == 8.5
    src.write_text("// kernel source, changed\n")
    assert bench.traffic_per_update() is None
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(tmp_path / "missing.cu"))
    assert bench.traffic_per_update() is None
