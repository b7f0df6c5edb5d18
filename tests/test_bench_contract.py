"""bench.py's output contract, on the CPU: the reference arm's JSON line (the
CPU oracle, timed on the headline workload with the GPU arm's metric and
unit), its silence on ranks other than 0, the one-line answer of the
configurations that have no reference arm, and the clock summary's reading of
nvidia-smi rows."""
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT


def run_bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          timeout=300, env=e, cwd=ROOT)


def one_line(r):
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_line_matches_the_gpu_arms_metric():
    import bench

    d = one_line(run_bench("--impl", "reference", "--steps", "2", "--warmup", "1"))
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "tasks/s" and d["higher_is_better"] is True
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["value"] > 0 and d["ms_per_step"] > 0
    w, desc = bench.workload("sgemm512", 0, 0)
    assert d["config"]["workload"] == desc
    assert (d["config"]["ranks"], d["config"]["tasks_per_rank"]) == (16, 64)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["vs_baseline"] is None


def test_reference_arm_vector_add_config():
    d = one_line(run_bench("--impl", "reference", "--workload", "vadd_tiny", "--steps", "1", "--warmup", "0"))
    assert d["config"]["ranks"] == 4 and d["config"]["tasks_per_rank"] == 8 and d["value"] > 0


def test_reference_arm_prints_nothing_on_other_ranks():
    r = run_bench("--impl", "reference", "--steps", "1", "--warmup", "0", env={"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.strip() == ""


@pytest.mark.parametrize("workload", ["grouped", "stress", "serving"])
def test_configs_without_a_reference_arm_say_so(workload):
    d = one_line(run_bench("--impl", "reference", "--workload", workload))
    assert d["impl"] == "reference" and d["unavailable"]


def test_clock_summary_reads_throttle_reasons():
    import bench

    s = bench.ClockSampler(0)
    assert s.summary() is None
    idle = ["0", "2070", "2070", "700.5", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    capped = ["0", "1980", "2070", "1399.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"]
    hot = ["0", "1500", "2070", "1200.0", "0x40", "Not Active", "Active", "Not Active", "Not Active"]
    s.rows = [idle, capped, idle]
    got = s.summary()
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0 and got["samples"] == 3
    assert got["reasons"] == ["sw_power_cap"]
    s.rows = [hot, capped]
    assert s.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s.summary()["sm_mhz"] == 1740.0
