"""Host logic of bench.py on CPU: clock-sample parsing, per-class rooflines, traffic
per launch and the peak-file fallback.  No GPU and no library calls."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _clock_line(mhz, mx, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if nm in reasons else "Not Active" for nm in names]
    return ", ".join(["0", str(mhz), str(mx), "900.5", "0x0"] + flags) + "\n"


def test_clock_summary_median_max_and_reasons(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write(_clock_line(2070, 2070))
        f.write(_clock_line(1965, 2070, ("sw_power_cap",)))
        f.write(_clock_line(2070, 2070))
        f.write("garbage line\n")
        f.write("0, [N/A], 2070, 1, 0, a, b, c, d\n")   # unparsable clock value: skipped
    c.proc = object()                                   # as if nvidia-smi had run
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_clock_summary_without_sampler():
    c = bench.Clocks(0)
    c.proc = None
    assert c.summary()["reasons"] == ["unavailable"]


def _prof(ms, calls, bytes_, flops):
    return {"ms": ms, "calls": calls, "bytes": bytes_, "flops": flops}


PEAKS = {"hbm": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "measured"}


def test_tensor_core_fp64_classes_against_bf16_peak():
    # 2 TFLOP/s of FP64-equivalent work = 28 x 2 TFLOP/s of bf16 digit-plane products
    prof = {"gram64tc": _prof(100.0, 3, 1e9, 2e12 * 0.1)}
    out = bench.kernel_rooflines(prof, PEAKS)
    assert out["gram64tc"]["bound"] == "tensor"
    assert out["gram64tc"]["fp64_equiv_tflops"] == pytest.approx(2.0)
    assert out["gram64tc"]["achieved"] == pytest.approx(56.0)
    assert out["gram64tc"]["frac"] == pytest.approx(56.0 / 1700.0, abs=1e-4)


def test_kernel_rooflines_bounds_and_fractions():
    prof = {
        "spmm": _prof(100.0, 10, 340e9 * 0.1, 0.0),           # 340 GB/s
        "vc64": _prof(50.0, 5, 1e9, 0.5 * 1.25e12 * 0.05),    # half the FP64 rate
        # FP64 SpMM: 0.8 of the FP64 rate vs 0.1 of HBM -> reported against the FP64 rate
        "spmm64": _prof(10.0, 2, 0.1 * 6800e9 * 0.01, 0.8 * 1.25e12 * 0.01),
        "syev": _prof(30.0, 4, 0.0, 0.0),                      # no roof: skipped
        "gram": _prof(0.0, 0, 0.0, 0.0),                       # never launched: skipped
    }
    out = bench.kernel_rooflines(prof, PEAKS)
    assert set(out) == {"spmm", "vc64", "spmm64"}
    assert out["spmm"]["bound"] == "hbm" and out["spmm"]["unit"] == "GB/s"
    assert out["spmm"]["achieved"] == pytest.approx(340.0)
    assert out["spmm"]["frac"] == pytest.approx(340.0 / 6800.0, abs=1e-4)
    assert out["vc64"]["bound"] == "alu" and out["vc64"]["frac"] == pytest.approx(0.5, abs=1e-4)
    assert out["spmm64"]["bound"] == "alu" and out["spmm64"]["frac"] == pytest.approx(0.8, abs=1e-4)
    assert out["vc64"]["calls"] == 5 and out["vc64"]["ms"] == 50.0


def test_spmm64_reported_against_hbm_when_that_fraction_is_larger():
    prof = {"spmm64": _prof(10.0, 1, 0.9 * 6800e9 * 0.01, 0.2 * 1.25e12 * 0.01)}
    out = bench.kernel_rooflines(prof, PEAKS)
    assert out["spmm64"]["bound"] == "hbm"
    assert out["spmm64"]["frac"] == pytest.approx(0.9, abs=1e-4)


def test_traffic_per_launch_scales_algorithmic_bytes():
    prof = _prof(1.0, 4, 4e8, 0.0)
    r = bench.TRAFFIC_RATIO["q1_64"]["spmm"]
    assert bench.traffic_per_launch("q1_64", "spmm", prof) == round(r * 1e8)
    assert bench.traffic_per_launch("q1_64", "syev", prof) is None
    assert bench.traffic_per_launch("q1_64", "gram64tc", prof) is None   # not measured
    assert bench.traffic_per_launch("q1_64", "vc64", prof) is None       # kernel changed
    assert bench.traffic_per_launch("other_workload", "spmm", prof) is None
    assert bench.traffic_per_launch("q1_64", "spmm", _prof(1.0, 0, 0.0, 0.0)) is None


def test_measured_peaks_file_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    fb = bench.measured_peaks()
    assert (fb["hbm"], fb["bf16"], fb["source"]) == (6800.0, 1900.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({
        "hbm_gbs": 7000.5, "bf16_tflops": 1950.0, "bf16_tflops_sustained": 1701.0}))
    m = bench.measured_peaks()
    assert (m["hbm"], m["bf16"], m["bf16_sustained"], m["source"]) == \
        (7000.5, 1950.0, 1701.0, "measured")


def test_reference_arm_reports_its_own_step_time(monkeypatch):
    """The reference line's ms_per_step is what a step took; its value extrapolates the
    per-iteration time to a whole solve (start-up + iterations x per-iteration time)."""
    calls = iter([(10.0, 2.0, 3.0), (11.0, 2.5, 3.5), (12.0, 1.5, 4.0)])
    monkeypatch.setattr(bench, "oracle_sample", lambda cfg: next(calls))
    monkeypatch.setattr(bench, "oracle_iterations", lambda cfg: 30)

    class A:
        config, steps, warmup = "q1_64", 2, 1
    line = bench.run_reference(A(), 0, 1)
    assert line["impl"] == "reference" and line["steps"] == 2
    assert line["ms_per_step"] == pytest.approx(1e3 * 11.5)
    assert line["value"] == pytest.approx(2.0 + 3.75 * 30)
    assert line["cpu_baseline"]["sparse_threads"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert bench.run_reference(A(), 1, 2) is None        # only rank 0 prints


def test_table_workload_filter_rejects_unknown_names(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--table", "--workloads", "q1_64,nope"])
    with pytest.raises(SystemExit, match="unknown workload 'nope'"):
        bench.main()
