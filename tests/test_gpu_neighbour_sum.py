"""The constant-coefficient stencil's fixed-point neighbour sum, checked
against correctly rounded sums (math.fsum) on the device.

The sum is exact in a 64-bit window aligned to the largest term, then
rounded once; so where no bit of any term falls below the window (every
exponent within 7 binades of the largest) it equals math.fsum bit for bit,
and elsewhere it is within one rounding plus terms * 2^-59 of the largest
term.  Non-finite and extreme tuples take the sequential FP64 sum.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1905_01549_gb300 import binding
    return binding


def _tuples(rng, count, terms, spread, base=0):
    """Random signed terms whose exponents lie in [base - spread, base]."""
    m = rng.uniform(1.0, 2.0, size=(count, terms))
    e = base - rng.integers(0, spread + 1, size=(count, terms))
    s = rng.choice([-1.0, 1.0], size=(count, terms))
    return s * np.ldexp(m, e)


def _seq(v):
    out = v[:, 0].copy()
    for j in range(1, v.shape[1]):
        out = out + v[:, j]
    return out


@pytest.mark.parametrize("terms", [4, 6])
def test_equals_correct_rounding_when_nothing_is_cut(B, terms):
    rng = np.random.default_rng(11)
    for base in (0, -30, 200, -900):
        v = _tuples(rng, 20000, terms, 7, base)
        out = B.prcg_test_neighbour_sum(v)
        ref = np.array([math.fsum(t) for t in v])
        assert np.array_equal(out, ref), base


@pytest.mark.parametrize("terms", [4, 6])
def test_error_bound_with_wide_exponent_spread(B, terms):
    rng = np.random.default_rng(12)
    v = _tuples(rng, 50000, terms, 80)
    out = B.prcg_test_neighbour_sum(v)
    ref = np.array([math.fsum(t) for t in v])
    big = np.abs(v).max(axis=1)
    # one rounding of ours and one of fsum (2 ulp covers a binade change),
    # plus the bits cut below the window
    bound = 2 * np.spacing(np.abs(ref)) + terms * 2.0 ** -59 * 2 * big
    assert np.all(np.abs(out - ref) <= bound)
    # and more accurate than sequential FP64 addition
    err, err_seq = np.abs(out - ref), np.abs(_seq(v) - ref)
    assert err.mean() < err_seq.mean() and np.count_nonzero(err) < np.count_nonzero(err_seq)


def test_exact_cancellation_and_signed_zeros(B):
    rng = np.random.default_rng(13)
    a = _tuples(rng, 1000, 3, 60)
    v = np.concatenate([a, -a], axis=1)
    out = B.prcg_test_neighbour_sum(v)
    assert np.all(out == 0.0)
    # one nonzero term among zeros of both signs: that term exactly
    z = np.zeros((4, 6))
    z[:, 1] = -0.0
    z[:, 4] = [1.5, -2.0 ** -900, 3.0 ** 40, -7.0]
    assert np.array_equal(B.prcg_test_neighbour_sum(z), z[:, 4])


def test_specials_take_the_fp64_sum(B):
    inf, nan = math.inf, math.nan
    v = np.array([
        [1.0, inf, 2.0, 3.0, 4.0, 5.0],
        [1.0, inf, -inf, 3.0, 4.0, 5.0],
        [nan, 1.0, 2.0, 3.0, 4.0, 5.0],
        [0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
        [5e-324, 5e-324, 1e-310, -2e-310, 0.0, 3e-300],   # all below 2^-959
        [1.7e308, 1.7e308, 1.0, 0.0, 0.0, 0.0],           # would overflow
        [2.0 ** 1019, -2.0 ** 1019, 1.0, 0.0, 0.0, 0.0],  # beyond the window's range
    ])
    out = B.prcg_test_neighbour_sum(v)
    seq = _seq(v)
    assert math.isinf(out[0]) and out[0] > 0
    assert math.isnan(out[1]) and math.isnan(out[2])
    assert out[3] == 0.0
    assert np.array_equal(out[4:], seq[4:])


def test_terms_next_to_the_range_limits(B):
    """Largest exponents just inside [64, 2040] use the fixed-point path and
    stay exact; a subnormal beside them vanishes within the bound."""
    lo = np.ldexp(1.0, 64 - 1023)      # smallest magnitude of exponent field 64
    hi = np.ldexp(1.0, 2040 - 1023)    # largest exponent field accepted
    v = np.array([[lo, lo, lo, lo, lo, -lo],
                  [hi, hi, -hi, hi, 0.0, 0.0],
                  [lo, 5e-324, 0.0, 0.0, 0.0, 0.0]])
    out = B.prcg_test_neighbour_sum(v)
    assert out[0] == 4 * lo and out[1] == 2 * hi and out[2] == lo


def test_invalid_arguments(B):
    with pytest.raises(B.PrcgError):
        B.prcg_test_neighbour_sum(np.zeros((3, 5)))
    assert B.prcg_test_neighbour_sum(np.zeros((0, 6))).shape == (0,)
