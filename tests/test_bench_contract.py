"""The benchmark's output contract, checked on the CPU through its reference arm (the oracle on the
host cores): one JSON line with the metric, value, unit, timing and configuration keys, the
reference arm's own cpu_baseline and e2e objects, and no device work."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def reference_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--grid", "36x16x16", "--n-s", "1e6"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_line_has_the_contract_keys(reference_line):
    d = reference_line
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["data"] == "synthetic" and d["dtype"] == "f64"
    assert "workload" in d["config"]


def test_reference_line_describes_its_own_cpu_run(reference_line):
    d = reference_line
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_device_line_carries_roofline_clocks_and_e2e():
    from helpers import cuda_available
    if not cuda_available():
        pytest.skip("needs a CUDA device")
    r = subprocess.run([sys.executable, "bench.py", "--steps", "2", "--warmup", "3", "--n-s", "1e6", "--shards", "2",
                        "--grid", "72x32x32", "--no-cpu-baseline", "--no-forms"], cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")][-1])
    assert d["value"] > 0 and d["unit"] == "superphotons/s" and d["gpu_launches"] > 0
    rl = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rl, k
    assert rl["bound"] == "alu" and 0.0 < rl["frac"] <= 1.05
    assert set(("sm_mhz", "sm_max_mhz", "reasons")) <= set(d["clocks"])
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
