"""Failure detection on the GPU without a fault: bounded waits and guard bands.

The persistent solve's grid barriers poll a bounded number of times.  A test
hook makes one CTA skip one barrier: every CTA's wait then runs out, the
solve reports PRCG_ERR_TIMEOUT, and the same context solves correctly
afterwards.  Separately, every buffer of a context is followed by guard
bands that the tests check after all kinds of work.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("variant,barrier", [("pr", 0), ("pr", 7), ("hs", 5), ("pipe_pr", 12),
                                             ("cgcg", 6), ("gv", 9)])
def test_skipped_barrier_times_out_and_context_recovers(G, variant, barrier):
    import torch
    from paper_1905_01549_gb300 import binding
    prob = case("poisson3d_ragged")
    A = csr_matrix(prob)
    b = torch.from_numpy(prob.b).cuda()
    with make_solver(G, prob, "csr", "none") as S:
        binding.prcg_inject_barrier_skip(S.handle, cta=3, barrier=barrier, spin_limit=1 << 16)
        x = torch.full((S.n,), 7.0, dtype=torch.float64, device="cuda")
        with pytest.raises(G.PrcgError) as e:
            S.solve(b, x0=x, variant=variant, tol=1e-10, maxit=1000)
        assert e.value.code == binding.PRCG_ERR_TIMEOUT
        assert bool((x == 7.0).all())          # no result is written on an error
        res = S.solve(b, variant=variant, tol=0.0, maxit=20)   # the context still works
        ref = O.solve(variant, A, prob.b, tol=0.0, maxit=20)
        assert res.iters == 20 and rel(res.x.cpu().numpy(), ref.x) <= 1e-10
        assert S.check_guards() == 0


def test_guard_bands_intact_after_every_kind_of_work(G):
    import torch
    prob = case("varcoef2d_ragged")
    b = torch.from_numpy(prob.b).cuda()
    with make_solver(G, prob, "stencil", "jacobi") as S:
        for v in ("hs", "pr", "pipe_pr", "m", "pipe_m", "cgcg", "gv"):
            S.solve(b, variant=v, tol=1e-10, maxit=2000, true_relres=True, trace=True)
        S.solve_refined_fp32(b, tol=1e-8)
        from paper_1905_01549_gb300 import binding
        lam = torch.randn(S.n, dtype=torch.float64, device="cuda")
        binding.prcg_grad_faces(S.handle, lam, b, torch.empty(
            prob.face_array().size, dtype=torch.float64, device="cuda"))
        S.error_anorm(b, torch.zeros_like(b))
        assert S.check_guards() == 0
    dense = P.model_problem(77, 1.0, 10.0)
    with G.Solver.from_dense(dense.A, precond="jacobi") as S:
        for v in ("hs", "pr", "pipe_pr", "cgcg", "gv"):
            S.solve(dense.b, variant=v, tol=1e-10, maxit=500, true_relres=True)
        assert S.check_guards() == 0
