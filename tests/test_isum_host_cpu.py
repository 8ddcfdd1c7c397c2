"""The stencil kernels' integer-pipe helpers (csrc/prcg_isum.cuh), compiled
for the host and checked without a GPU: the fixed-point neighbour sum against
math.fsum (correct rounding of the exact sum) and the invariant-divisor
quotient against integer division.  The same source runs on the device; the
device side is checked by tests/test_gpu_neighbour_sum.py."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("isum") / "isum_host_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", out, os.path.join(HERE, "isum_host_check.cu")],
                   check=True, capture_output=True)
    return out


def _run_sum(exe, v, tmp_path):
    v = np.ascontiguousarray(v, dtype=np.float64)
    fin, fout = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(fin, "wb") as f:
        f.write(np.int32(v.shape[1]).tobytes())
        f.write(np.int64(v.shape[0]).tobytes())
        f.write(v.tobytes())
    subprocess.run([exe, "sum", str(fin), str(fout)], check=True)
    raw = open(fout, "rb").read()
    n = v.shape[0]
    out = np.frombuffer(raw[:8 * n], dtype=np.float64)
    fixed = np.frombuffer(raw[8 * n:], dtype=np.int8).astype(bool)
    return out, fixed


def _tuples(rng, count, terms, spread, base=0):
    m = rng.uniform(1.0, 2.0, size=(count, terms))
    e = base - rng.integers(0, spread + 1, size=(count, terms))
    s = rng.choice([-1.0, 1.0], size=(count, terms))
    return s * np.ldexp(m, e)


@pytest.mark.parametrize("terms", [4, 6])
def test_sum_is_correctly_rounded_when_nothing_is_cut(exe, tmp_path, terms):
    rng = np.random.default_rng(21)
    v = np.concatenate([_tuples(rng, 20000, terms, 7, base) for base in (0, -40, 300, -900)])
    out, fixed = _run_sum(exe, v, tmp_path)
    assert fixed.all()
    assert np.array_equal(out, np.array([math.fsum(t) for t in v]))


@pytest.mark.parametrize("terms", [4, 6])
def test_sum_error_bound_and_accuracy(exe, tmp_path, terms):
    rng = np.random.default_rng(22)
    v = _tuples(rng, 50000, terms, 80)
    out, fixed = _run_sum(exe, v, tmp_path)
    ref = np.array([math.fsum(t) for t in v])
    big = np.abs(v).max(axis=1)
    assert fixed.all()
    assert np.all(np.abs(out - ref) <= 2 * np.spacing(np.abs(ref)) + terms * 2.0 ** -58 * big)
    seq = v[:, 0].copy()
    for j in range(1, terms):
        seq = seq + v[:, j]
    assert np.abs(out - ref).mean() < np.abs(seq - ref).mean()


def test_sum_cancellation_specials_and_limits(exe, tmp_path):
    rng = np.random.default_rng(23)
    a = _tuples(rng, 500, 3, 60)
    out, _ = _run_sum(exe, np.concatenate([a, -a], axis=1), tmp_path)
    assert np.all(out == 0.0)
    lo, hi = np.ldexp(1.0, 64 - 1023), np.ldexp(1.0, 2040 - 1023)
    v = np.array([[math.inf, 1, 2, 3, 4, 5], [math.nan, 1, 2, 3, 4, 5], [0.0] * 6,
                  [3e-300, 1e-310, 0, 0, 0, 0], [1.7e308, 1.7e308, 1, 0, 0, 0],
                  [lo, lo, lo, lo, lo, -lo], [hi, hi, -hi, hi, 0, 0], [lo, 5e-324, 0, 0, 0, 0],
                  [1.5, -0.0, 0.0, -0.0, 0.0, 0.0]])
    out, fixed = _run_sum(exe, v, tmp_path)
    assert list(fixed) == [False, False, False, False, False, True, True, True, True]
    assert math.isinf(out[0]) and math.isnan(out[1]) and out[2] == 0.0
    assert out[3] == 3e-300 + 1e-310 and math.isinf(out[4])
    assert out[5] == 4 * lo and out[6] == 2 * hi and out[7] == lo and out[8] == 1.5


@pytest.mark.parametrize("d", [1, 2, 3, 7, 13, 24, 45, 97, 160, 255, 256, 257, 1000, 4097,
                               65535, 65536, 65537, (1 << 20) + 1, 46341, (1 << 30) + 3,
                               (1 << 31) - 1])
def test_invariant_divisor_quotient(exe, d):
    n = (1 << 31) - 1
    r = subprocess.run([exe, "div", str(d), str(n)], check=True, capture_output=True, text=True)
    bad, checked = (int(t) for t in r.stdout.split())
    assert checked > (1 << 22) and bad == 0
