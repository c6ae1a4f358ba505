"""Host logic of bench.py (no GPU): the clock summary taken from nvidia-smi's
CSV samples, and the use of the committed ncu summary for the roofline's
traffic (only while the kernel source it was taken on is unchanged, and only
for the workload it was taken on)."""
import os

import pytest


def test_clock_summary_from_samples(tmp_path):
    import bench
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1390.2, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    open(s.path, "w").write("\n".join(rows) + "\n")
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    assert not os.path.exists(s.path)          # the sample file is removed


def test_clock_summary_without_samples(tmp_path):
    import bench
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "none.csv")
    assert s.summary() is None


def test_profile_traffic_needs_the_same_kernel_source_and_workload(tmp_path, monkeypatch):
    import bench
    prof = tmp_path / "prof.md"
    prof.write_text(f"# summary\n\nkernel_source_hash: {bench.kernel_source_hash()}\n"
                    f"dram_bytes_per_launch_full: 4044593920\n")
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profile_traffic() == pytest.approx(4044593920.0)
    assert bench.profile_traffic("ls_4000x50000_f32") is None
    prof.write_text("kernel_source_hash: 0000000000000000\ndram_bytes_per_launch_full: 1\n")
    assert bench.profile_traffic() is None
