"""Host logic of the benchmark line on CPU: the roofline denominators and
algorithmic work per unit, the clock-record parsing, and the rule that DRAM
traffic is reported only while the measured kernel's sources are unchanged."""
import json
import math
import os
import sys
import types

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_flops_per_cell_update_of_the_batched_disk():
    # P = 128, C = 1976 (R = 50 nm at a = 2 nm): two field evaluations per Heun step
    P, C = 128, 1976
    per_eval = bench.fft_flops_per_eval(P, C)
    # six real 2D transforms of 2.5 P^2 log2 P^2 flops, the tensor multiply, the epilogue
    assert per_eval == pytest.approx(6 * 2.5 * P * P * 14 + 14 * P * 65 + 60 * C)
    assert 2 * per_eval / C == pytest.approx(3720.32, abs=0.01)


def test_fp32_peak_from_unit_counts():
    assert bench.fp32_alu_peak_tflops(152) == pytest.approx(80.54784)
    assert bench.fp32_alu_peak_tflops(152, sm_mhz=1000.0) == pytest.approx(152 * 128 * 2 * 1e9 / 1e12)


def test_hbm_bytes_per_cell_update_of_the_large_disk():
    # 8 replicas of R = 500 nm: D = 500, C = 196,364, P = 1024
    wl = types.SimpleNamespace(P=1024, B=8, C=196364, D=500)
    per_step = bench.global_path_bytes_per_step(wl)
    kh = 513
    per_eval = 8 * (60 * 196364 + 4 * 3 * 500 * kh * 8) + kh * kh * 16
    assert per_step == 2 * per_eval * bench.CHUNK
    assert per_step / (8 * 196364 * bench.CHUNK) == pytest.approx(376.16, abs=0.01)


def _write_clocks(path, rows):
    with open(path, "w") as f:
        for r in rows:
            f.write(", ".join(r) + "\n")


def test_clock_record_median_and_reasons(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    s.proc = object()   # sampled (no nvidia-smi here): summary() only reads the file
    row = lambda sm, swp="Not Active", hw="Not Active": ["0", sm, "2070", "900.5", "0x0", hw, "Not Active",
                                                       "Not Active", swp]
    _write_clocks(s.path, [row("2070"), row("2055", swp="Active"), row("1995"), ["garbled"], row("2070")])
    out = s.summary()
    assert out["samples"] == 4
    assert out["sm_mhz"] == pytest.approx((2055 + 2070) / 2)
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    _write_clocks(s.path, [row("1500", hw="Active")])
    assert s.summary()["reasons"] == ["hw_slowdown"]
    _write_clocks(s.path, [])
    assert s.summary()["reasons"] == ["unsampled"]


def test_unsampled_clock_record():
    s = bench.ClockSampler(0)
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_traffic_is_reported_only_for_unchanged_kernel_sources(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "kernel_traffic.json")) as f:
        entries = json.load(f)["entries"]
    for workload, e in entries.items():
        assert e["dram_bytes_per_launch"] > 0
        monkeypatch.setattr(bench, "kernel_sources_sha256", lambda w=workload, h=e["sources_sha256"]: h)
        assert bench.profiled_traffic(workload) == e["dram_bytes_per_launch"]
        monkeypatch.setattr(bench, "kernel_sources_sha256", lambda w=workload: "0" * 64)
        assert bench.profiled_traffic(workload) is None
    assert bench.profiled_traffic("no such workload") is None


def test_kernel_source_hash_covers_every_listed_file():
    for workload, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_1207_2192_gb300", "csrc", f)), (workload, f)
    h = bench.kernel_sources_sha256("large_disk")
    assert len(h) == 64
    assert bench.kernel_sources_sha256("large_disk") == h
    assert bench.kernel_sources_sha256("plain") == bench.kernel_sources_sha256("batched_heun")


def test_measured_peaks_or_fallback():
    p = bench.measured_peaks()
    assert p["hbm_gbs"] > 1000.0
    assert math.isfinite(p["hbm_gbs"])
