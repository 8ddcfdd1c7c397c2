"""Exact-arithmetic pins for the oracle (rational arithmetic, fractions.Fraction).

Section 1 of the paper: every variant is mathematically equivalent to HS-CG,
so in exact arithmetic all of them produce HS-CG's iterates x_k, r_k and
scalars alpha_k, beta_k.  HS-CG itself is pinned by finite termination
(k distinct eigenvalues -> r_k = 0 at some step <= k) and by the exact
solution from brute-force rational Gaussian elimination.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import problems as P

VARIANTS = O.VARIANTS


def _exact_solve(A, b):
    """Gaussian elimination in rationals (brute force on tiny inputs)."""
    n = len(b)
    M = [[A[i, j] for j in range(n)] + [b[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * bb for a, bb in zip(M[r], M[c])]
    return np.array([M[i][n] / M[i][i] for i in range(n)], dtype=object)


def _case(seed, n):
    rng = np.random.default_rng(seed)
    A = P.random_int_spd(n, rng)
    b = P.fraction_vector(rng.integers(-5, 6, size=n))
    if not any(b):
        b[0] = Fraction(1)
    return A, b


@pytest.mark.parametrize("seed,n", [(1, 4), (2, 5), (3, 6), (4, 7), (5, 8)])
@pytest.mark.parametrize("precond", [False, True])
def test_all_variants_reproduce_hs_exactly(seed, n, precond):
    A, b = _case(seed, n)
    d = O.jacobi_inverse_diagonal(A) if precond else None
    x0 = P.fraction_vector(np.random.default_rng(seed + 100).integers(-2, 3, size=n))
    ref = O.hs_cg(A, b, x0=x0, d=d, record=n + 1)
    assert ref.status == O.OK and ref.iters <= n
    for v in VARIANTS:
        res = O.solve(v, A, b, x0=x0, d=d, record=n + 1)
        assert res.status == O.OK, v
        assert res.iters == ref.iters, v
        for k, ((xa, ra), (xb, rb)) in enumerate(zip(ref.iterates, res.iterates)):
            assert all(xa == xb) and all(ra == rb), (v, k)
        for k in range(1, ref.iters + 1):
            assert res.scalars[k]["alpha"] == ref.scalars[k]["alpha"], (v, k)
            if "beta" in ref.scalars[k] and "beta" in res.scalars[k]:
                assert res.scalars[k]["beta"] == ref.scalars[k]["beta"], (v, k)


@pytest.mark.parametrize("precond", [False, True])
def test_predicted_scalars_equal_recomputed_exactly(precond):
    """nu'_k (Eq. 2.3, and M-CG's form) equals <r~_k, r_k> in exact arithmetic."""
    A, b = _case(11, 7)
    d = O.jacobi_inverse_diagonal(A) if precond else None
    for v in ("pr", "pipe_pr", "m", "pipe_m"):
        res = O.solve(v, A, b, d=d)
        for k in range(1, res.iters + 1):
            sc = res.scalars[k]
            assert sc["nu_pred"] == sc["nu"], (v, k)


def test_ablations_are_exactly_equivalent_too():
    """Without recompute the recurrences are still exact (Eq. 3.17, Fig. 2 legend)."""
    A, b = _case(7, 6)
    ref = O.hs_cg(A, b, record=10)
    for res in (O.pr_cg(A, b, recompute_nu=False, record=10),
                O.pipe_pr_cg(A, b, recompute_w=False, record=10)):
        assert res.iters == ref.iters
        for (xa, ra), (xb, rb) in zip(ref.iterates, res.iterates):
            assert all(xa == xb) and all(ra == rb)


@pytest.mark.parametrize("eigs", [[1, 1, 2, 2, 3, 3, 3], [2, 5, 5, 5, 5, 9], [4, 4, 4, 4, 4]])
def test_finite_termination_distinct_eigenvalues(eigs):
    rng = np.random.default_rng(len(eigs) + sum(eigs))
    A = P.int_spd_with_eigs(eigs, rng)
    b = P.fraction_vector(rng.integers(1, 6, size=len(eigs)))
    kdistinct = len(set(eigs))
    xs = _exact_solve(A, b)
    for v in VARIANTS:
        res = O.solve(v, A, b, maxit=len(eigs) + 2)
        assert res.status == O.OK, v
        assert res.iters <= kdistinct, (v, res.iters)
        assert all(res.x == xs), v


@pytest.mark.parametrize("seed,n", [(21, 5), (22, 8)])
def test_exact_solution_matches_gaussian_elimination(seed, n):
    A, b = _case(seed, n)
    xs = _exact_solve(A, b)
    for precond in (False, True):
        d = O.jacobi_inverse_diagonal(A) if precond else None
        for v in VARIANTS:
            res = O.solve(v, A, b, d=d)
            assert res.status == O.OK and res.iters <= n
            assert all(res.x == xs), (v, precond)
            assert all(A.dot(res.x) == b)


def test_zero_rhs_and_exact_start():
    A, b = _case(31, 5)
    z = P.fraction_vector([0] * 5)
    for v in VARIANTS:
        res = O.solve(v, A, z)
        assert res.iters == 0 and res.status == O.OK and all(res.x == z)
        xs = _exact_solve(A, b)
        res = O.solve(v, A, b, x0=xs)
        assert res.iters == 0 and res.status == O.OK
