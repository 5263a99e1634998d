"""Host-side logic of bench.py (CPU): the clock record, the traffic record,
and the reference arm's JSON line on a small sample."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_summary_parses_nvidia_smi_lines():
    cs = bench.ClockSampler(0)
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    cs.lines = [
        "0, 1410, 2070, 1365.2, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1500, 2070, 1370.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1380, 2070, 1350.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    s = cs.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 1410.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["power_w"] == 1365.2
    cs.lines = ["0, 900, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active"]
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    cs.lines = []
    assert cs.summary()["samples"] == 0


def test_traffic_record_only_for_its_workload_and_source(monkeypatch):
    import hashlib
    import os
    w = dict(bench.TRAFFIC_RECORD["workload"])
    with open(os.path.join(bench.ROOT, bench.TRAFFIC_RECORD["source"]), "rb") as f:
        current = hashlib.sha256(f.read()).hexdigest()
    # the record counts only while the kernel source is the one it was taken with
    want = bench.TRAFFIC_RECORD["bytes_per_launch"] \
        if current == bench.TRAFFIC_RECORD["sha256"] else None
    assert bench.recorded_traffic(w) == want
    monkeypatch.setitem(bench.TRAFFIC_RECORD, "sha256", current)
    assert bench.recorded_traffic(w) == bench.TRAFFIC_RECORD["bytes_per_launch"]
    for key, other in (("n", 4096), ("k", 1), ("tile_band", 16), ("precision", "dual_bf16")):
        assert bench.recorded_traffic(dict(w, **{key: other})) is None
    monkeypatch.setitem(bench.TRAFFIC_RECORD, "sha256", "0" * 64)
    assert bench.recorded_traffic(w) is None


def test_algorithmic_flops():
    # D0 layer of the dual forms: (2 + 3K) 2 n^3
    assert bench.alg_flops_layers(8192, 3, 1) == 11 * 2.0 * 8192 ** 3
    assert bench.alg_flops_layers(100, 1, 4) == 4 * 5 * 2.0 * 100 ** 3


def test_reference_arm_line(tmp_path):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", "--oracle-n", "128"],
                         capture_output=True, text=True, timeout=600, env=env, cwd=tmp_path)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["value"] > 0 and line["unit"] == "TFLOP/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "TFLOP/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
