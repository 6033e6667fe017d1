"""The benchmark's reference arm (the FP64 oracle timed on the host) on CPU:
every workload prints one JSON line with the contract's keys, the same
metric and unit as the workload's own arm, an oracle CPU baseline, and an
e2e object with no host-device bytes.  Small sizes keep each run to a few
seconds."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


@pytest.mark.parametrize("workload,metric_key,unit", [
    ("clustered256", "force", "pairs/s"), ("centers256", "centers256", "pairs/s"),
    ("pm256", "pm256", "particles/s"), ("fof256", "fof256", "particles/s"),
    ("step256", "step256", "particles/s"), ("diff64", "diff64", "pairs/s")])
def test_reference_arm_line(workload, metric_key, unit):
    sys.path.insert(0, ROOT)
    import bench
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          workload, "--steps", "1", "--warmup", "0", "--n-particles", "4096"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d)
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRICS[metric_key]
    assert d["unit"] == unit and d["higher_is_better"] is True
    assert d["value"] > 0
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == d["value"] and cpu["cores"] >= 1 and cpu["sample"]
    assert "cpu_model" in cpu
    assert d["e2e"] == {"value": d["value"], "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == workload
