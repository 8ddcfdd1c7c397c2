"""The oracle's per-iteration work against Table 1's printed costs
(tests/golden/table1_costs.txt): inner products (scal) and matrix-vector
products per iteration of every variant.  A dropped or an extra inner
product, or a recompute left out (pipe-PR-CG's second product), changes the
count.  Counted as the difference between k + 1 and k iterations, so
initialize() is excluded."""
import numpy as np
import pytest

import oracle as O
import oracle.cg_variants as CV
from golden import table1

TABLE1 = table1()


def _counts(variant, A, b, d, k):
    nd, na = [0], [0]
    saved = CV._dot

    def dot(u, v):
        nd[0] += 1
        return saved(u, v)

    def apply(x):
        na[0] += 1
        return A @ x

    CV._dot = dot
    try:
        res = O.solve(variant, apply, b, d=d, tol=0.0, maxit=k)
    finally:
        CV._dot = saved
    assert res.iters == k
    return nd[0], na[0]


def _system():
    rng = np.random.default_rng(17)
    B = rng.standard_normal((24, 24))
    return B @ B.T + 24 * np.eye(24), rng.standard_normal(24)


def test_fixture_lists_every_variant():
    assert set(TABLE1) == set(O.VARIANTS)


@pytest.mark.parametrize("variant", O.VARIANTS)
def test_inner_products_and_products_per_iteration(variant):
    A, b = _system()
    d5, a5 = _counts(variant, A, b, None, 5)
    d6, a6 = _counts(variant, A, b, None, 6)
    assert d6 - d5 == TABLE1[variant]["scal"], (variant, d6 - d5)
    assert a6 - a5 == TABLE1[variant]["products"], (variant, a6 - a5)


@pytest.mark.parametrize("variant", O.VARIANTS)
def test_jacobi_adds_only_the_stopping_norm(variant):
    """With a preconditioner the oracle adds one inner product per iteration
    where the stopping test needs <r, r> and the algorithm's own sums do not
    already hold it (the stopping rule is a reading, Table 1 does not count
    it); the products are unchanged."""
    A, b = _system()
    d = 1.0 / np.diag(A)
    d5, a5 = _counts(variant, A, b, d, 5)
    d6, a6 = _counts(variant, A, b, d, 6)
    assert d6 - d5 in (TABLE1[variant]["scal"], TABLE1[variant]["scal"] + 1), (variant, d6 - d5)
    assert a6 - a5 == TABLE1[variant]["products"]
