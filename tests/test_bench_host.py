"""Host-side logic of bench.py (no GPU): the clock/throttle summary the timing rules depend on, the
algorithmic flop counts of the roofline, the workload description, the seeded pixel sample, and the
JSON line of the reference arm (the CPU oracle)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_1209_6038_gb300 import inputs  # noqa: E402


def sampler_with(rows):
    s = bench.ClockSampler(0)
    s.proc = object()  # as if nvidia-smi were running
    with open(s.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    return s


def test_clock_summary_reads_median_clock_and_throttle_reasons():
    s = sampler_with([
        "0, 2070, 2070, 240.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 250.3, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1800, 2070, 260.0, 0x8, Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    try:
        out = s.summary()
    finally:
        os.remove(s.path)
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["power_w_max"] == 260.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_flop_counts_per_step_attempt():
    # DP5(4): 6 new right-hand sides + 362; RK4: 4 + 102; radial ordinary rays are straight (0 per RHS)
    assert bench.flops_per_step(0, 1, 1) == 6 * 36 + 362
    assert bench.flops_per_step(1, 1, 1) == 6 * 30 + 362
    assert bench.flops_per_step(1, 0, 0) == 4 * 34 + 102
    assert bench.flops_per_step(0, 0, 1) == 362


def test_workload_config_names_the_full_workload():
    cfg = bench.workload_config(inputs.FULL)
    assert cfg["images"] == 12 and cfg["width"] == 1920 and cfg["height"] == 1080 and cfg["spp"] == 4
    assert cfg["integrator"] == "dp45" and cfg["tol"] == 1e-9
    assert inputs.FULL.rays == 12 * 1920 * 1080 * 4


def test_pixel_sample_is_seeded_sorted_and_distinct():
    w = inputs.FULL
    a = bench.sample_pixels(w, 3, 500)
    b = bench.sample_pixels(w, 3, 500)
    c = bench.sample_pixels(w, 4, 500)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.all(np.diff(a) > 0) and a.min() >= 0 and a.max() < w.width * w.height


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-pixels", "16"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "rays/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
