"""bench.py's reference arm on CPU: the C oracle timed on the host cores.

The arm prints one JSON line with the same metric, unit and direction as
the GPU arm, `impl` = "reference", a `cpu_baseline` describing the run and
an `e2e` object with no host-device copies; under a multi-process launch
only rank 0 runs and prints.  A small grid keeps the run short.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, args=()):
    env = dict(os.environ)
    env.update(extra_env or {})
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "poisson3d_20",
           "--steps", "2", "--warmup", "1", *args]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_line():
    import bench
    res = _run()
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "iters/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "poisson3d_20_csr_jacobi_pr"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["cores"] == len(os.sched_getaffinity(0))
    assert "stands in" not in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_print_nothing():
    res = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, ("--gpus", "2"))
    assert res.returncode == 0, res.stderr[-2000:]
    assert not [l for l in res.stdout.splitlines() if l.startswith("{")]


def test_reference_rank0_reports_the_job_size():
    res = _run({"RANK": "0", "WORLD_SIZE": "2", "LOCAL_RANK": "0"}, ("--gpus", "2", "--op", "stencil"))
    assert res.returncode == 0, res.stderr[-2000:]
    d = json.loads([l for l in res.stdout.splitlines() if l.startswith("{")][0])
    assert d["n_gpus"] == 2
    assert "stands in" in d["cpu_baseline"]["sample"]
