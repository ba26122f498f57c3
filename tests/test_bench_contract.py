"""The benchmark's reference arm runs on the host alone (the FP64 oracle),
so its JSON line can be checked on the CPU: one line, every key of the
contract, the oracle described as the CPU baseline, and no host-device
traffic counted for it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_complete_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--ref-side", "10"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "elements/s" and d["higher_is_better"] is True
    assert d["dtype"] == "f64" and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the line describes the benchmark's workload, the 256^3 lattice, and the
    # sample each step timed; the time per step is the sample's, as timed
    assert d["config"]["n_masses"] == 256 ** 3 and d["config"]["n_springs"] == 216338940
    assert "10^3" in d["config"]["sample"] and "10^3" in cb["sample"]
    assert d["extrapolated_ms_per_step_at_workload"] > d["ms_per_step"]
