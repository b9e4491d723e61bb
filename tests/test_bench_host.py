"""Host logic of bench.py that needs no GPU: the clock summary over the timed window, the
roofline arithmetic, the scaling of the stored DRAM traffic, and the reference arm's JSON line
(the plain CPU oracle on a tiny sample of the workload)."""
import argparse
import json
import math

import pytest

import bench


def _line(sm, smax=2070, reasons=("Not Active",) * 4):
    return f"0, {sm}, {smax}, 900.5, 0x0000000000000000, " + ", ".join(reasons)


def test_clock_summary_takes_the_timed_window():
    lines = [(0.90, _line(1200)), (1.00, _line(2070)), (1.05, _line(2055)),
             (1.10, _line(2070, reasons=("Not Active", "Not Active", "Not Active", "Active"))),
             (1.30, _line(345))]  # before and after the window: idle clocks
    s = bench.ClockSampler.summary(lines, 0.95, 1.20, 50)
    assert s["samples"] == 3 and s["window"] == "timed region"
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_throttle_reasons_by_name():
    act = ("Active", "Not Active", "Active", "Not Active")
    s = bench.ClockSampler.summary([(1.0, _line(1500, reasons=act))], 0.5, 1.5, 50)
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1500.0


def test_clock_summary_falls_back_to_the_next_sample():
    """A window shorter than the sampling interval may hold no sample: the first one after its
    start stands for it, and the line says so."""
    lines = [(0.90, _line(1000)), (1.08, _line(2040)), (1.20, _line(300))]
    s = bench.ClockSampler.summary(lines, 1.00, 1.02, 50)
    assert s["samples"] == 1 and s["window"] == "next sample" and s["sm_mhz"] == 2040.0


def test_clock_summary_skips_malformed_lines():
    lines = [(1.0, "No devices were found"), (1.1, "0, [N/A], 2070, 1, 0, a, b, c, d"), (1.2, _line(1980))]
    s = bench.ClockSampler.summary(lines, 0.0, 2.0, 50)
    assert s["samples"] == 1 and s["sm_mhz"] == 1980.0


def test_clock_sampler_that_never_started():
    s = bench.ClockSampler(0).stop()
    assert s["sm_mhz"] is None and s["reasons"] == ["nvidia-smi unavailable"]


def test_roofline_of_the_modelled_kernel_with_the_largest_time():
    n = 512 ** 3
    rep = {"sweep_L0": (16, 16 * 0.5), "residual": (2, 2 * 2.0), "exchange": (1, 3.4), "unmodelled": (1, 50.0)}
    peaks = {"hbm_gbs": 6000.0, "source": "measured"}
    r = bench.roofline(rep, n, "mixed", peaks, {"sweep_L0": 2.5e9})
    assert r["kernel"] == "sweep_L0" and r["bound"] == "hbm" and r["launches"] == 16
    assert r["achieved"] == pytest.approx(16 * n / 0.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert r["traffic"] == 2.5e9 and r["algorithmic_bytes_per_launch"] == 16 * n
    assert r["share_of_traced_ms"] == pytest.approx(8.0 / (8.0 + 4.0 + 3.4 + 50.0))
    assert bench.roofline({}, n, "mixed", peaks, {}) is None
    assert bench.roofline({"unmodelled": (1, 1.0)}, n, "mixed", peaks, {}) is None


def test_stored_traffic_scales_with_the_cells():
    with open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    full = bench.load_traffic(512, t["precision"])
    half = bench.load_traffic(256, t["precision"])
    assert set(full) == set(t["scopes"])
    for k, v in t["scopes"].items():
        n0 = v.get("captured_n", t["captured_n"])
        assert full[k] == pytest.approx(v["dram_bytes_per_launch"] * (512 / n0) ** 3)
        assert half[k] == pytest.approx(full[k] / 8)
    other = "fp64" if t["precision"] == "mixed" else "mixed"
    assert bench.load_traffic(512, other) == {}


def _ref_args(**kw):
    a = dict(gpus=1, steps=1, warmup=0, n=512, precision="mixed", rtol=1e-8, oracle_n=16)
    a.update(kw)
    return argparse.Namespace(**a)


def test_reference_arm_prints_one_line_on_rank_zero(capsys):
    assert bench.run_reference(_ref_args(), 1, 0) == 0
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    line = json.loads(out[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 0
    assert line["value"] > 0 and math.isfinite(line["value"])
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == 1 and "16^3" in line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["grid"] == [512] * 3


def test_reference_arm_other_ranks_exit_without_work(capsys):
    assert bench.run_reference(_ref_args(), 2, 1) == 0
    assert capsys.readouterr().out == ""
