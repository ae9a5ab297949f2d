"""Host logic of bench.py that decides what a benchmark line reports (no GPU): the clock
record parsed from nvidia-smi samples, the measured peaks, and the roofline entry's
choice of dominant kernel and its algorithmic flops per launch."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _summary(tmp_path, text):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write(text)
    return s.summary()


def test_clock_summary_reads_median_max_and_active_reasons(tmp_path):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap (csv, noheader, nounits)
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2055, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = _summary(tmp_path, "\n".join(rows) + "\n")
    assert r["samples"] == 3
    assert r["sm_mhz"] == 2055 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]  # "Not Active" is not a reason


def test_clock_summary_reports_thermal_and_hw_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active",
            "0, 1600, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active"]
    r = _summary(tmp_path, "\n".join(rows) + "\n")
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert r["sm_mhz"] == 1550


def test_clock_summary_without_samples_says_unavailable(tmp_path):
    r = _summary(tmp_path, "")
    assert r["samples"] == 0 and r["sm_mhz"] is None and r["reasons"] == ["unavailable"]


def test_measured_peaks_come_from_the_measured_file():
    """The HBM peak is the measured copy bandwidth in MEASURED_PEAKS.json when that file is
    present, else the stated fallback (6.8 TB/s, labelled as such)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    got, src = bench.measured_peaks()
    if os.path.exists(path):
        with open(path) as f:
            want = float(json.load(f)["hbm_gbs"])
        assert src == "measured" and got == want
    else:
        assert src == "fallback" and got == 6800.0


def test_roofline_takes_the_kernel_with_the_most_time():
    ncell = 2048 * 2048
    per_dir = bench.flops_per_cell_rhs() / 2.0
    prof = {"sweep_x_lx_2d": (60, 6.6), "sweep_y_stage_2d": (60, 6.5), "dt_from_maxima": (20, 0.2),
            "reduce": (0, 0.0)}
    r = bench.roofline_of(prof, ncell, "f64", 80.0, "derived")
    assert r["kernel"] == "sweep_x_lx_2d" and r["bound"] == "alu"
    assert r["launch_ms"] == pytest.approx(0.11)
    assert r["flops_per_launch"] == pytest.approx(ncell * per_dir)  # one direction, no stage update
    assert r["achieved"] == pytest.approx(ncell * per_dir / 0.11e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 80.0)
    assert r["traffic"] is None  # counters are stored for the single-precision kernels only
    prof["sweep_y_stage_2d"] = (60, 6.7)
    r = bench.roofline_of(prof, ncell, "f64", 80.0, "derived")
    assert r["kernel"] == "sweep_y_stage_2d"
    assert r["flops_per_launch"] == pytest.approx(ncell * (per_dir + 20))  # plus the stage update


def test_roofline_of_the_banded_stage_counts_both_directions():
    ncell = 2048 * 2048
    per_dir = bench.flops_per_cell_rhs() / 2.0
    r = bench.roofline_of({"stage_band_2d": (60, 18.0), "dt_from_maxima": (20, 0.2)}, ncell, "f64", 80.0, "x")
    assert r["kernel"] == "stage_band_2d"
    assert r["flops_per_launch"] == pytest.approx(ncell * (2 * per_dir + 20))
