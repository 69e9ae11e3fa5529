"""Host-side logic of bench.py on the CPU: the reference arm's JSON line (the CPU
oracle timed on a bounded sample), the summary of the clock record taken during the
timed region, the check that a stored DRAM-traffic figure belongs to the current
kernel source, and the fallback peaks."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

LINE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"}


def _bench(*argv, env=None):
    e = dict(os.environ, OMP_NUM_THREADS="2")
    e.update(env or {})
    return subprocess.run([sys.executable, "bench.py", *argv], cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_line():
    r = _bench("--impl", "reference", "--n", "96", "--steps", "2", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert LINE_KEYS | {"impl", "cpu_baseline", "e2e"} <= set(d)
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["dtype"] == "f64"
    assert d["value"] > 0 and abs(d["ms_per_step"] * d["value"] - 1e3) < 1e-6 * 1e3
    assert "workload" in d["config"] and d["config"]["n"] == 96
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "sampled output columns" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_stay_silent():
    r = _bench("--impl", "reference", "--n", "96", "--steps", "1", "--warmup", "0",
               env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


class _Stopped:
    """Stands in for the nvidia-smi process once its output has been read."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _summary(rows, window=None):
    """rows: (seconds after t=1000, the fields after the timestamp)."""
    import datetime
    c = bench.ClockSampler(0)
    c.proc = _Stopped()
    c.lines = []
    for t, rest in rows:
        stamp = datetime.datetime.fromtimestamp(1000.0 + t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        c.lines.append((0.0, stamp + ", " + rest))
    return c.stop(None if window is None else (1000.0 + window[0], 1000.0 + window[1]))


IDLE = "Not Active, Not Active, Not Active, Not Active"


def test_clock_summary_takes_median_and_reasons():
    out = _summary([
        (0.00, "0, 2070, 2070, 812.3, 0x0000000000000000, " + IDLE),
        (0.03, "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"),
        (0.06, "0, 2055, 2070, 1200.0, 0x0000000000000000, " + IDLE),
        (0.07, "malformed line"),
        (0.08, "0, [N/A], 2070, 0, 0x0, Active, Not Active, Not Active, Not Active"),
    ])
    assert out == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}


def test_clock_summary_names_every_slowdown():
    out = _summary([
        (0.0, "0, 1500, 2070, 1400.0, 0x48, Active, Active, Not Active, Not Active"),
        (0.1, "0, 1600, 2070, 1400.0, 0x20, Not Active, Not Active, Active, Not Active"),
    ])
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1550.0 and out["samples"] == 2


def test_clock_summary_keeps_the_timed_window():
    rows = [(0.00, "0, 1200, 2070, 300.0, 0x1, " + IDLE),       # idle, before the region
            (0.50, "0, 2070, 2070, 1300.0, 0x0, " + IDLE),
            (0.55, "0, 2040, 2070, 1350.0, 0x0, " + IDLE),
            (0.60, "0, 2070, 2070, 1380.0, 0x0, " + IDLE),
            (1.50, "0, 1100, 2070, 200.0, 0x1, Active, Not Active, Not Active, Not Active")]
    out = _summary(rows, window=(0.45, 0.65))
    assert out["samples"] == 3 and out["in_window"] is True and out["sm_mhz"] == 2070.0
    assert out["reasons"] == [] and abs(out["window_ms"] - 200.0) < 1e-6
    near = _summary(rows, window=(0.70, 0.72))      # no sample inside: the nearest 250 ms
    assert near["in_window"] is False and near["samples"] == 3


def test_clock_summary_without_nvidia_smi():
    c = bench.ClockSampler(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_clock_sampler_reads_a_running_tool(tmp_path, monkeypatch):
    """The sampler as bench.py runs it, against a stand-in nvidia-smi on PATH that
    prints a timestamped sample every 10 ms."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text(
        "#!" + sys.executable + "\n"
        "import datetime, sys, time\n"
        "while True:\n"
        "    t = datetime.datetime.now().strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]\n"
        "    print(t + ', 0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active',"
        " flush=True)\n"
        "    time.sleep(0.01)\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    import time
    c = bench.ClockSampler(0)
    c.start()
    assert c.lines, "no first sample before the timed region"
    t0 = time.time()
    time.sleep(0.2)
    t1 = time.time()
    time.sleep(0.05)
    out = c.stop((t0, t1))
    assert out["in_window"] is True and out["samples"] >= 5
    assert out["sm_mhz"] == 2070.0 and out["reasons"] == []


def test_recorded_traffic_belongs_to_its_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1707_08369_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = b"// output stage\n"
    (csrc / "svdup_mixed.cu").write_bytes(src)
    rec = {"n": 8192, "mode": "bf16x3", "bytes_per_launch": 404239168,
           "source_sha256": hashlib.sha256(src).hexdigest()}
    (tmp_path / "profiles" / "umma_out_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic(8192, "bf16x3") == 404239168
    assert bench.recorded_traffic(4096, "bf16x3") is None      # another workload
    assert bench.recorded_traffic(8192, "fp64") is None        # another mode
    (csrc / "svdup_mixed.cu").write_bytes(src + b"// changed\n")
    assert bench.recorded_traffic(8192, "bf16x3") is None      # kernel changed since


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk, src = bench.load_peaks()
    assert src == "fallback"
    assert pk == {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def test_measured_peaks_are_read_when_present():
    if not os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        pytest.skip("no measured peaks in this checkout")
    pk, src = bench.load_peaks()
    assert src == "measured"
    assert pk["hbm_gbs"] > 0 and pk["bf16_tflops"] > 0 and pk["bf16_tflops_sustained"] > 0


def test_fp64_peak_from_unit_counts():
    # 152 SMs x 2 DFMA per SM per clock x 2 flops at 2070 MHz
    assert abs(bench.fp64_peak_tflops(2070.0) - 1.25856) < 1e-9
    assert bench.fp64_peak_tflops(None) == bench.fp64_peak_tflops(2070.0)


def test_roofline_uses_the_algorithmic_count_of_the_dominant_kernel():
    """frac = App. D's algorithmic flops of the dominant kernel's launches over their
    summed event time and the peak; the executed and useful figures ride beside it."""
    # stage: (ms, launches, useful flops, executed flops, algorithmic flops)
    kern = {"p2m": (0.5, 4, 1e9, 6e9, 4e9), "m2l": (0.25, 4, 2e9, 12e9, 1e10),
            "out": (2.0, 4, 3e11, 1.8e12, 1.4e10)}
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
    r = bench.roofline_of(kern, 1, {"sm_mhz": 2070.0}, peaks, "fallback", 8192, "bf16x3")
    assert r["kernel"] == "k_umma<OUT>" and r["bound"] == "tensor" and r["launches"] == 4
    per_launch_s = 2.0 / 4 / 1e3
    assert abs(r["achieved"] - 1.4e10 / 4 / per_launch_s / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1700.0) < 1e-12
    assert abs(r["executed_tflops"] - 1.8e12 / 4 / per_launch_s / 1e12) < 1e-9
    assert "fallback" in r["peak_source"]
    r64 = bench.roofline_of(kern, 0, {"sm_mhz": 1035.0}, peaks, "measured", 8192, "fp64")
    assert r64["kernel"] == "k_gemm_f64<OUT>" and r64["bound"] == "alu"
    assert abs(r64["peak"] - bench.fp64_peak_tflops(1035.0)) < 1e-12
    assert abs(r64["frac"] - r64["achieved"] / r64["peak"]) < 1e-12
