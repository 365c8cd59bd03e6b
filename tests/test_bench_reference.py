"""The benchmark's reference arm (the oracle on the host cores) prints one
JSON line with the keys the benchmark contract asks for, for the 2D and 3D
workloads, and an `unavailable` line for the workloads it does not cover."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", *extra], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("extra,sites", [((), 64 ** 3), (("--workload", "prec1024"), 256 * 256),
                                         (("--workload", "prec1024", "--stencil", "isotropic"), 256 * 256)])
def test_reference_line(extra, sites):
    line = _run(*extra)
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["config"]["sites_per_step"] == sites
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["warmup"] >= 3 and line["steps"] == 1


def test_reference_unavailable_for_batched_workloads():
    line = _run("--workload", "ens96")
    assert line["impl"] == "reference" and "unavailable" in line
