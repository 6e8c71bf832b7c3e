"""Host-side logic of bench.py that needs no GPU: the clock sampler's summary of nvidia-smi lines
(median SM clock under load, maximum clock, throttle reasons seen), and the byte and flop
constants of the roofline."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    return s.summary()


def test_clock_summary_median_max_and_reasons():
    # index, clocks.sm, clocks.max.sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 910.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _sampler(lines)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_ignores_malformed_lines():
    lines = ["garbage", "0, [N/A], 2070, 1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1800, 2070, 1200, 0x40, Not Active, Active, Not Active, Not Active"]
    s = _sampler(lines)
    assert s["sm_mhz"] == 1800.0 and s["reasons"] == ["hw_thermal_slowdown"]
    assert _sampler([])["reasons"] == ["unsampled"]


def test_roofline_constants():
    # 2 DFMA per clock per SM x 2 flops x 152 SMs x 2.07 GHz
    assert abs(bench.FP64_PEAK_TFLOPS - 1258.56) < 1e-6
    # the unit-diagonal 7-point stencil: 6 neighbour multiply-adds + the dot product's per component
    assert bench.SPMV_FLOPS_PER_CELL == 3 * 14
    # x, r, p read and written once: 6 passes of a 3-component vector
    assert bench.PCG_BYTES_PER_CELL == {"fp64": 144, "fp32": 72}
    assert bench.PC2_LINE_BYTES_PER_CELL == 7 * 3 * 8 + 8


def test_reference_arm_line_on_host_cores():
    # the reference arm runs the oracle's OpenMP timing build on every host core, names the grid it
    # ran and the source of its iteration count, and times one thread beside it
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--grid", "12x12x24",
                          "--steps", "1", "--warmup", "0", "--no-anchors", "--ref-iters", "50"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"]["grid"] == "12x12x24"
    cpu = line["cpu_baseline"]
    assert cpu["cores"] == (os.cpu_count() or 1) and cpu["iters_per_step"] == 50
    assert cpu["single_thread_value"] > 0 and line["value"] > 0
    assert "count given" in cpu["iters_source"]


def test_full_oracle_step_anchor_has_its_model_beside_it():
    a = bench.oracle_full_step("parity_32x32x64", "16x16x32", threads=2)
    assert a["threads"] == 2 and a["pcg_iters"] > 0 and a["ms"] > 0 and a["sampled_model_ms"] > 0
