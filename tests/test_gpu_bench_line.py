"""bench.py's JSON line on a small case (GPU): the keys and the arithmetic
that tie them together.  The 48^3 system fits in L2, which the line must
say; the default 256^3 run is the measured one."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_small_case():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    cmd = [sys.executable, "bench.py", "--workload", "poisson3d_48", "--steps", "3", "--warmup", "3",
           "--no-extras"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["metric"] == bench.METRIC and d["unit"] == "iters/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["scaling"] == "weak"
    cfg = d["config"]
    assert cfg["workload"] == "poisson3d_48_csr_jacobi_pr" and cfg["n"] == 48 ** 3
    assert "fit in the 129 MB L2" in cfg["l2"]
    K = cfg["iters_per_solve"]
    assert K > 0
    # value = iterations of the timed solves / their device time
    assert abs(d["value"] - 3 * K / (d["ms_per_step"] * 3 / 1e3)) <= 1e-6 * d["value"]
    roof = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in roof
    assert roof["bound"] in ("hbm", "alu") and roof["peak"] > 0
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) <= 1e-9 * max(1.0, roof["frac"])
    assert roof["traffic"] is None        # recorded for the 256^3 workload only
    assert [s["kernel"] for s in roof["sweeps"]] == ["k_pr_a", "k_pr_b"]
    assert d["gpu_launches"] > 0
    clk = d["clocks"]
    assert {"sm_mhz", "sm_max_mhz", "reasons", "samples"} <= set(clk)
    assert clk["samples"] == 0 or clk["sm_max_mhz"] > 0
