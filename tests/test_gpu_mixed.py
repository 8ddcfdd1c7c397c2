"""FP32-inner / FP64-refinement solver vs the FP64 oracle and the mixed oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import problems as P
from gpu_common import case, csr_matrix, make_solver, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


@pytest.mark.parametrize("name", ["poisson2d_64", "poisson3d_ragged", "varcoef3d_ragged",
                                  "poisson3d_nx24"])
@pytest.mark.parametrize("op", ["csr", "stencil"])
@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_mixed_reaches_fp64_tolerance(G, name, op, precond):
    import torch
    prob = case(name)
    A = csr_matrix(prob)
    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
    ref = O.pr_cg(A, prob.b, d=d, tol=1e-13, maxit=20 * prob.n)     # the FP64 answer
    xm, st_m, outer_m, inner_m, hist_m = O.refined_fp32(A, prob.b, tol=1e-8, d=d)
    with make_solver(G, prob, op, precond) as S:
        x, status, outer, inner, trr, hist, ms = S.solve_refined_fp32(
            torch.from_numpy(prob.b).cuda(), tol=1e-8, inner_tol=1e-4)
    assert status == G.PRCG_OK and st_m == O.OK
    assert trr <= 1e-8 and O.true_relres(A, prob.b, x.cpu().numpy()) <= 1.5e-8
    kappa_est = 1e4 if name.startswith("varcoef") and precond == "none" else 1e3
    assert rel(x.cpu().numpy(), ref.x) <= 1e-8 * kappa_est
    assert abs(outer - outer_m) <= 1, (outer, outer_m)
    assert np.all(np.diff(hist) < 0)


def test_mixed_strakos_diagonal(G):
    import torch
    lam, b = P.strakos_diagonal(100000, 1e-3, 1e3, 0.8)
    n = len(lam)
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    with G.Solver.from_csr(rp, ci, lam) as S:
        x, status, outer, inner, trr, hist, ms = S.solve_refined_fp32(
            torch.from_numpy(b).cuda(), tol=1e-8, inner_tol=1e-4)
    xs = np.full(n, 1 / np.sqrt(n))
    assert status == G.PRCG_OK and trr <= 1e-8
    assert rel(x.cpu().numpy(), xs) <= 1e-8 * 1e6
    xm, st_m, outer_m, _, _ = O.refined_fp32(sp.diags(lam, format="csr"), b, tol=1e-8)
    assert abs(outer - outer_m) <= 1


def test_mixed_zero_rhs_and_csr_fallback(G):
    import torch
    with G.Solver.from_stencil((9, 7)) as S:
        x = torch.ones(63, dtype=torch.float64, device="cuda")
        x, status, outer, inner, trr, hist, ms = S.solve_refined_fp32(
            torch.zeros(63, dtype=torch.float64, device="cuda"), x0=x)
        assert status == G.PRCG_OK and outer == 0 and float(x.abs().max()) == 0.0
