"""The multi-threaded C oracle (oracle/cg_oracle.c) against the numpy oracle.

The C oracle times the CPU baseline on every host core.  It is a second,
independent transcription of Algorithms 1-3 (plain FP64 loops, OpenMP
reductions), so it is pinned here to the numpy oracle, whose own pins are
exact arithmetic, Cholesky, the rounding-gap bounds and the paper's tables:
over the first 20 iterations of well-conditioned systems the two agree to
1e-12 relative in x_k and ||r_k|| / ||b|| for every variant, with and
without Jacobi, on 1 and 4 threads; solved to 1e-10 they stop within one
iteration of each other.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import problems as P
from oracle import c_oracle as C


def _cases():
    return {"poisson2d_64": P.poisson2d_64(),
            "poisson3d_ragged": P.grid_problem((21, 13, 11), "t_p3r"),
            "shifted2d": P.grid_problem((33, 47), "t_sh2", shift=0.05, rhs="uniform"),
            "varcoef3d_jacobi": P.grid_problem((19, 11, 7), "t_vc3r", sigma=2.0)}


CASES = _cases()


def _A(prob):
    rp, ci, v = prob.csr
    return sp.csr_matrix((v, ci, rp), shape=(prob.n, prob.n))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant", ["hs", "pr", "pipe_pr"])
@pytest.mark.parametrize("threads", [1, 4])
def test_c_oracle_matches_numpy_oracle(name, variant, threads):
    prob = CASES[name]
    A = _A(prob)
    pcs = ("jacobi",) if name == "varcoef3d_jacobi" else ("none", "jacobi")
    for pc in pcs:
        d = O.jacobi_inverse_diagonal(A) if pc == "jacobi" else None
        ref = O.solve(variant, A, prob.b, d=d, tol=0.0, maxit=20)
        res = C.solve(variant, prob.csr, prob.b, d=d, tol=0.0, maxit=20, threads=threads,
                      history=True)
        assert res.status == ref.status == O.NOT_CONVERGED and res.iters == 20
        assert np.linalg.norm(res.x - ref.x) / np.linalg.norm(ref.x) <= 1e-12, (pc,)
        h = np.asarray(ref.hist)
        assert np.all(np.abs(res.hist - h) <= 1e-12 * h), (pc,)
        ref = O.solve(variant, A, prob.b, d=d, tol=1e-10, maxit=4 * prob.n)
        res = C.solve(variant, prob.csr, prob.b, d=d, tol=1e-10, maxit=4 * prob.n, threads=threads)
        assert res.status == ref.status == O.OK and abs(res.iters - ref.iters) <= 1
        assert O.true_relres(A, prob.b, res.x) <= 1e-9


def test_c_oracle_special_cases():
    prob = CASES["poisson2d_64"]
    A = _A(prob)
    for v in ("hs", "pr", "pipe_pr"):
        res = C.solve(v, prob.csr, np.zeros(prob.n), tol=1e-10, maxit=50)   # b = 0
        assert res.status == O.OK and res.iters == 0
        res = C.solve(v, prob.csr, prob.b, tol=1e-10, maxit=0)
        assert res.status == O.NOT_CONVERGED and res.iters == 0
        bad = prob.b.copy()
        bad[3] = np.nan
        ref = O.solve(v, A, bad, tol=1e-10, maxit=50)
        res = C.solve(v, prob.csr, bad, tol=1e-10, maxit=50)
        assert res.status == ref.status == O.BREAKDOWN and res.iters == ref.iters == 0
    with pytest.raises(ValueError):
        C.solve("pr", prob.csr, prob.b, tol=-1.0)
    assert C.max_threads() >= 1
