"""bench.py's reference arm (the FP64 oracle on the host cores) on workloads that need no GPU to
generate their inputs: one JSON line with impl = reference, the arm's metric and unit, a positive
throughput, the oracle named as the baseline, and no host-device traffic."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["block", "adjoint"])
def test_reference_line(workload):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "0", "--block", "4"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "slices/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["metric"].startswith("slices/s")
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["ms_per_step"] == pytest.approx(1e3 / line["value"])
    assert workload.split()[0] in line["config"]["workload"]
