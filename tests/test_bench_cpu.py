"""bench.py's reference arm (the FP64 oracle on the host) keeps the JSON-line
contract: one line, the headline metric and unit, the workload config, a
cpu_baseline and an e2e object describing the same run.  Runs on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-sample", "4"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "rollout-steps/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["config"]["K"] == 8192 and d["config"]["T"] == 100 and d["config"]["L"] == 512
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_warmup_below_three_is_refused():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "2"], capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert out.returncode != 0 and "warmup" in (out.stderr + out.stdout)


def test_plant_step_roofline_counts_one_read_of_the_records():
    """The plant step's algorithmic bytes are one read of the 12 outputs' FP32
    field-pair records (1376 B per pair, ceil(L/2) pairs per output), and its
    fraction is the achieved bandwidth over the HBM peak given."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.plant_step_roofline([0.02, 0.02], 512, {"hbm_gbs": 6000.0}, "tc")
    assert r["bytes_per_launch"] == 12 * 256 * 1376
    assert abs(r["achieved"] - 12 * 256 * 1376 / 0.02e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-12
    assert r["bound"] == "hbm" and r["launches_per_step"] == 3
    assert bench.plant_step_roofline([0.01], 513, {}, "fp32")["bytes_per_launch"] == 12 * 257 * 1376


def test_tensor_peak_follows_the_clock_record():
    """The tensor roofline divides by the measured burst bf16 rate unless the run's
    clock record shows it held down by the power cap (sw_power_cap and a median SM
    clock below 95 % of the maximum), where the seconds-long sustained rate applies."""
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"bf16_tflops": 1788.7, "bf16_tflops_sustained": 1393.1}
    assert bench.tensor_peak(peaks, {"reasons": [], "sm_mhz": 2032.0, "sm_max_mhz": 2032.0})[0] == 1788.7
    capped = {"reasons": ["sw_power_cap"], "sm_mhz": 1432.0, "sm_max_mhz": 2032.0}
    assert bench.tensor_peak(peaks, capped)[0] == 1393.1
    # the cap flagged in a few samples while the clock stayed at its maximum: burst
    flagged = {"reasons": ["sw_power_cap"], "sm_mhz": 2021.0, "sm_max_mhz": 2032.0}
    assert bench.tensor_peak(peaks, flagged)[0] == 1788.7
    assert bench.tensor_peak(peaks, None)[0] == 1788.7


def test_clock_scaled_tensor_peak():
    """The clock-scaled view divides by the burst rate times the run's median clock over
    the maximum, and is absent without a clock record."""
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"bf16_tflops": 1788.7}
    v = bench.clock_scaled(peaks, {"sm_mhz": 1016.0, "sm_max_mhz": 2032.0}, 447.175)
    assert abs(v["peak"] - 894.35) < 1e-9 and abs(v["frac"] - 0.5) < 1e-12
    assert bench.clock_scaled(peaks, None, 1.0) is None
