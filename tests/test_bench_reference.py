"""The benchmark's reference arm (`bench.py --impl reference`): the oracle
timed on the host cores, no GPU needed.  Its JSON line carries the same
metric and unit as the GPU arm of the same workload, the oracle's own
timing as `cpu_baseline`, and an end-to-end record with no host-device
copies."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1", *extra],
                         capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


@pytest.mark.parametrize("workload", [None, "batch"])
def test_reference_arm_line(workload):
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    d = _reference_line(*(["--workload", workload] if workload else []))
    assert d["impl"] == "reference"
    assert d["unit"] == "descriptors/s" and d["higher_is_better"] is True
    if workload is None:
        assert d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["data"] == "synthetic" and "workload" in d["config"]
