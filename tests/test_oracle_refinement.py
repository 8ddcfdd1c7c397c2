"""Pins for the mixed-precision oracle (FP32 inner PR-CG, FP64 refinement).

Classical iterative-refinement theory fixes what it must do: each outer step
contracts the true residual by about max(inner_tol, c * kappa * u_32), so it
reaches an FP64-level tolerance that a pure FP32 solve cannot, as long as
kappa * u_32 < 1."""
import numpy as np
import scipy.sparse as sp

import oracle as O
import problems as P

U32 = 2.0 ** -24


def test_refinement_reaches_fp64_tolerance_on_strakos_diagonal():
    lam, b = P.strakos_diagonal(20000, 1e-3, 1e3, 0.8)
    A = sp.diags(lam, format="csr")
    x, status, outer, inner, hist = O.refined_fp32(A, b, tol=1e-8, inner_tol=1e-4)
    assert status == O.OK and hist[-1] <= 1e-8
    xs = np.full(20000, 1 / np.sqrt(20000))
    kappa = 1e6
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-8 * kappa
    # contraction per step: at most ~max(inner_tol, kappa u32) (plus slack)
    rate = max(1e-4, kappa * U32)
    for a, b_ in zip(hist, hist[1:]):
        assert b_ <= 20 * rate * a


def test_pure_fp32_solve_stalls_but_refinement_does_not():
    prob = P.grid_problem((24, 24), "t_mx")
    rp, ci, v = prob.csr
    A = sp.csr_matrix((v, ci, rp), shape=(prob.n, prob.n))
    r32 = O.pr_cg(A.astype(np.float32), prob.b.astype(np.float32), tol=1e-10, maxit=5000)
    x32 = r32.x.astype(np.float64)
    assert O.true_relres(A, prob.b, x32) > 1e-8          # FP32 alone cannot get there
    x, status, outer, inner, hist = O.refined_fp32(A, prob.b, tol=1e-11)
    assert status == O.OK and O.true_relres(A, prob.b, x) <= 1e-11
    assert 1 <= outer <= 6


def test_refinement_zero_rhs():
    A = sp.diags(np.arange(1.0, 11.0), format="csr")
    x, status, outer, inner, hist = O.refined_fp32(A, np.zeros(10))
    assert status == O.OK and not x.any() and outer == 0
