"""The benchmark's reference arm runs on the host cores (it times the FP64
oracle), so its output line can be checked here without a GPU: one JSON line
with the keys and types the harness reads, a cpu_baseline describing the run
and an e2e entry with no host-device traffic."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "mc32",
           "--steps", "1", "--warmup", "0", "--ref-samples", "4", *extra]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def check_line(d):
    for k, t in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                 ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                 ("dtype", str), ("data", str), ("config", dict)):
        assert isinstance(d[k], t), k
    assert d["impl"] == "reference" and d["vs_baseline"] is None
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_line():
    d = run_reference()
    check_line(d)
    assert d["config"]["workload"].startswith("mc32: 32x32 grid")


def test_reference_arm_paper_field_and_w_cycle():
    """The Matern Phi_2 field and the W-cycle reach the oracle and the workload name."""
    d = run_reference("--field", "phi2", "--cycle", "2")
    check_line(d)
    assert "Phi_2" in d["config"]["workload"] and "cycle index 2" in d["config"]["workload"]
