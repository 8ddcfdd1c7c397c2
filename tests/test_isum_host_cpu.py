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


# ---------------------------------------------------------------------------
# block fixed point with one scale per vector (to_fixed / fixed_to_double)

def _round_half_away(fr):
    """round(fr) with half-way cases away from zero, fr a Fraction."""
    from fractions import Fraction
    a = abs(fr)
    q = int(a + Fraction(1, 2))   # floor(|x| + 1/2)
    return q if fr >= 0 else -q


def _run_fx(exe, v, S, tmp_path):
    v = np.ascontiguousarray(v, dtype=np.float64)
    fin, fout = tmp_path / "fin.bin", tmp_path / "fout.bin"
    with open(fin, "wb") as f:
        f.write(np.int32(v.shape[1]).tobytes())
        f.write(np.int64(v.shape[0]).tobytes())
        f.write(np.int32(S).tobytes())
        f.write(v.tobytes())
    subprocess.run([exe, "fx", str(fin), str(fout)], check=True)
    raw = open(fout, "rb").read()
    n = v.shape[0]
    out = np.frombuffer(raw[:8 * n], dtype=np.float64)
    sums = np.frombuffer(raw[8 * n:16 * n], dtype=np.int64)
    bad = np.frombuffer(raw[16 * n:], dtype=np.int8).astype(bool)
    return out, sums, bad


@pytest.mark.parametrize("S", [58, 0, -300, 400, 900])
def test_block_fixed_point_is_exact_integer_arithmetic(exe, tmp_path, S):
    """Each P_j is v_j 2^S rounded half away from zero, the sum of the P_j is
    exact, and the conversion back is the correctly rounded acc 2^-S (Python's
    Fraction -> float rounds to nearest even): bit-equal on random tuples
    whose magnitudes span 70 binades below the window top 2^(58 - S)."""
    from fractions import Fraction
    rng = np.random.default_rng(1000 + S)
    count, K = 3000, 6
    top = 58 - S
    e = top - 1 - rng.integers(0, 70, size=(count, K))
    m = rng.uniform(1.0, 2.0, size=(count, K)) * rng.choice([-1.0, 1.0], size=(count, K))
    v = np.ldexp(m, e)
    v[::7, 0] = 0.0
    out, sums, bad = _run_fx(exe, v, S, tmp_path)
    assert not bad.any()
    scale = Fraction(2) ** S if S >= 0 else Fraction(1, 2 ** (-S))
    for t in range(count):
        acc = sum(_round_half_away(Fraction(x) * scale) for x in v[t])
        assert int(sums[t]) == acc, t
        assert out[t] == float(Fraction(acc) / scale), t


def test_block_fixed_point_error_bound_and_window(exe, tmp_path):
    """The converted sum is within K 2^-(S+1) plus one rounding of the exact
    sum; values at or above 2^(58 - S), infinities and NaN are flagged."""
    S = 40
    rng = np.random.default_rng(5)
    v = np.ldexp(rng.uniform(-1, 1, size=(2000, 6)), 17)   # below 2^18 = 2^(58 - S)
    out, _, bad = _run_fx(exe, v, S, tmp_path)
    assert not bad.any()
    exact = np.array([math.fsum(r) for r in v])
    assert np.all(np.abs(out - exact) <= 6 * 2.0 ** -(S + 1) + np.abs(exact) * 2.0 ** -53)
    edge = np.array([[2.0 ** 18, 0, 0, 0, 0, 0], [np.inf, 0, 0, 0, 0, 0], [np.nan, 1, 0, 0, 0, 0],
                     [2.0 ** 18 * (1 - 2.0 ** -53), 0, 0, 0, 0, 0]])
    _, _, bad = _run_fx(exe, edge, S, tmp_path)
    assert list(bad) == [True, True, True, False]


def test_fixed_scale_and_magnitude_bound(exe, tmp_path):
    """fixed_scale(B) is the largest S with B 2^S < 2^58; amax_bound of the
    high word of |B| is an upper bound of |B| within a factor 1 + 2^-19."""
    rng = np.random.default_rng(6)
    B = np.ldexp(rng.uniform(1.0, 2.0, 3000), rng.integers(-880, 880, 3000))
    B = np.concatenate([B, [0.0, np.inf, np.nan, 2.0 ** -950, 2.0 ** 950]])
    fin, fout = tmp_path / "sin.bin", tmp_path / "sout.bin"
    with open(fin, "wb") as f:
        f.write(np.int64(len(B)).tobytes())
        f.write(B.tobytes())
    subprocess.run([exe, "scale", str(fin), str(fout)], check=True)
    raw = open(fout, "rb").read()
    sc = np.frombuffer(raw[:4 * len(B)], dtype=np.int32)
    bd = np.frombuffer(raw[4 * len(B):], dtype=np.float64)
    for b, s_, u in zip(B[:3000], sc[:3000], bd[:3000]):
        assert math.ldexp(b, int(s_)) < 2.0 ** 58 <= math.ldexp(b, int(s_) + 1)
        assert b < u <= b * (1 + 2.0 ** -19)
    assert list(sc[3000:]) == [-100000] * 5
