"""The bench's JSON line: the keys and units the measurement contract fixes,
for the reference arm (the CPU oracle, no GPU) and for the CUDA arm."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
             "scaling", "vs_baseline", "dtype", "data", "config", "e2e"}


def run_bench(*args, timeout=600):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    r = run_bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert BASE_KEYS <= set(r)
    assert r["impl"] == "reference"
    assert r["steps"] == 1 and r["warmup"] == 3 and r["value"] > 0
    assert r["cpu_baseline"]["kind"] == "oracle" and r["cpu_baseline"]["cores"] >= 1
    assert r["cpu_baseline"]["value"] == r["value"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert r["config"]["workload"]


@pytest.mark.gpu
def test_cuda_arm_line():
    # enough steps for the clock sampler (one sample per 200 ms) to see the timed region
    r = run_bench("--steps", "300", "--warmup", "3", "--no-forms", "--no-cpu")
    assert BASE_KEYS <= set(r)
    assert r["n_gpus"] == 1 and r["steps"] == 300 and r["warmup"] == 3
    assert r["higher_is_better"] is True and r["value"] > 0
    assert r["gpu_launches"] > 0
    roof = r["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(roof)
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-9
    e2e = r["e2e"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0 and e2e["value"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(r["clocks"])
    assert r["config"]["workload"]
