"""The allocation-free PR-CG entry point against the regular one and the oracle.

prcg_pr_solve_stencil_noalloc exists for callers that cannot allocate
device memory (foreign memory pools, real-time loops without cudaMalloc);
it keeps its iteration vectors in a fixed file-scope device array.  Here it
is called through the C ABI twice in a row (the second call must not see the
first call's leftovers) and compared with prcg_solve and with the oracle's
PR-CG (Algorithm 2) on the same inputs, including the branches of its own
code: b = 0, maxit = 0, an exact x_0, a NaN in b and a breakdown.
This file sorts last so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import oracle as O
import problems as P
from gpu_common import csr_matrix, rel

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10       # first iterations, as in the parity tests
CONVERGED_TOL = 1e-7   # converged x, as in the parity tests


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


@pytest.mark.parametrize("dims,shift", [((64, 64), 0.0), ((21, 13, 11), 0.0), ((33, 47), 0.05),
                                        ((256, 256), 0.0)])
@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_noalloc_matches_regular_entry_point(G, dims, shift, precond):
    import torch
    from paper_1905_01549_gb300 import binding
    pc = binding.PRCG_PRECOND_JACOBI if precond == "jacobi" else binding.PRCG_PRECOND_NONE
    nx, ny = dims[0], dims[1]
    nz = dims[2] if len(dims) == 3 else 1
    regular = G.Solver.from_stencil(dims, diag_shift=shift, precond=precond)
    try:
        for call, tag in enumerate(("first", "second")):
            prob = P.grid_problem(dims, f"noalloc_{tag}", shift=shift, with_csr=False)
            b = torch.from_numpy(prob.b).cuda()
            for tol, maxit, bar in ((0.0, 20, ITER_TOL), (1e-10, 4 * prob.n, CONVERGED_TOL)):
                x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
                hist = torch.full((maxit + 1,), -1.0, dtype=torch.float64, device="cuda")
                status, iters = binding.prcg_pr_solve_stencil_noalloc(
                    len(dims), nx, ny, nz, shift, pc, b, x, tol, maxit, hist)
                ref = regular.solve(b, variant="pr", tol=tol, maxit=maxit, history=True)
                assert status == ref.status, (call, tol)
                assert abs(iters - ref.iters) <= max(1, int(0.05 * ref.iters)), (call, iters, ref.iters)
                assert rel(x.cpu().numpy(), ref.x.cpu().numpy()) <= bar, (call, tol)
                h = hist.cpu().numpy()[:iters + 1]
                m = min(len(h), len(ref.hist))
                assert np.allclose(h[:m], ref.hist[:m], rtol=1e-9 if tol == 0 else 1e-6, atol=0)
                if tol == 0.0:
                    # the oracle's PR-CG, Algorithm 2, on the same inputs
                    A = csr_matrix(P.grid_problem(dims, "noalloc_op", shift=shift))
                    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
                    orc = O.solve("pr", A, prob.b, d=d, tol=0.0, maxit=maxit)
                    assert status == orc.status and iters == orc.iters
                    assert rel(x.cpu().numpy(), orc.x) <= ITER_TOL, (call, "oracle")
                    assert np.allclose(h, orc.hist, rtol=1e-9, atol=0)
    finally:
        regular.close()


def _noalloc(G, dims, b, x, tol, maxit, precond="none"):
    from paper_1905_01549_gb300 import binding
    import torch
    pc = binding.PRCG_PRECOND_JACOBI if precond == "jacobi" else binding.PRCG_PRECOND_NONE
    nz = dims[2] if len(dims) == 3 else 1
    hist = torch.full((maxit + 1,), -1.0, dtype=torch.float64, device="cuda")
    status, iters = binding.prcg_pr_solve_stencil_noalloc(len(dims), dims[0], dims[1], nz, 0.0, pc,
                                                          b, x, tol, maxit, hist)
    return status, iters, hist.cpu().numpy()[:iters + 1]


def test_noalloc_special_cases_match_oracle_and_regular(G):
    """The branches the single-CTA kernel handles itself, each called twice."""
    import torch
    dims = (8, 8)
    prob = P.grid_problem(dims, "noalloc_edge")
    A = csr_matrix(prob)
    b = torch.from_numpy(prob.b).cuda()
    with G.Solver.from_stencil(dims) as S:
        for _ in range(2):
            # b = 0 with a nonzero x_0: x = 0, K = 0 (the library's reading; the
            # oracle from x_0 = 0 stops at K = 0 with x = 0 as well)
            x = torch.ones(prob.n, dtype=torch.float64, device="cuda")
            st, k, _ = _noalloc(G, dims, torch.zeros_like(x), x, 1e-10, 100)
            xr = torch.ones_like(x)
            ref = S.solve(torch.zeros_like(x), x0=xr, variant="pr", tol=1e-10, maxit=100)
            orc = O.solve("pr", A, np.zeros(prob.n), tol=1e-10, maxit=100)
            assert st == ref.status == orc.status == G.PRCG_OK and k == ref.iters == orc.iters == 0
            assert float(x.abs().max()) == 0.0 and float(xr.abs().max()) == 0.0
            # maxit = 0: K = 0, x untouched
            x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
            st, k, h = _noalloc(G, dims, b, x, 1e-10, 0)
            orc = O.solve("pr", A, prob.b, tol=1e-10, maxit=0)
            assert st == orc.status == G.PRCG_NOT_CONVERGED and k == orc.iters == 0
            assert float(x.abs().max()) == 0.0 and np.allclose(h, orc.hist, rtol=1e-12)
            # x_0 the exact solution: K = 0
            xt = torch.from_numpy(prob.x_true).cuda()
            st, k, _ = _noalloc(G, dims, b, xt.clone(), 1e-12, 100)
            orc = O.solve("pr", A, prob.b, x0=prob.x_true.copy(), tol=1e-12, maxit=100)
            assert st == orc.status == G.PRCG_OK and k == orc.iters == 0
            # a NaN in b: ||b|| and nu_0 are NaN, the run breaks down after
            # initialize() (K = 0), as the oracle and prcg_solve do
            bn = prob.b.copy()
            bn[5] = np.nan
            x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
            st, k, _ = _noalloc(G, dims, torch.from_numpy(bn).cuda(), x, 1e-10, 50)
            orc = O.solve("pr", A, bn, tol=1e-10, maxit=50)
            ref = S.solve(torch.from_numpy(bn).cuda(), variant="pr", tol=1e-10, maxit=50)
            assert st == orc.status == ref.status == G.PRCG_BREAKDOWN and k == orc.iters == ref.iters


def test_noalloc_runs_past_convergence_in_bounded_time(G):
    """tol = 0 at the largest accepted maxit (4 n + 1000): once r_k is rounding
    noise the run either keeps iterating to maxit or stops on unusable
    scalars (BREAKDOWN, Section 3.1); which of the two, and when, depends on
    the order of the sums, so only the outcome's properties are checked."""
    import torch
    dims = (4, 4)
    prob = P.grid_problem(dims, "noalloc_brk")
    A = csr_matrix(prob)
    b = torch.from_numpy(prob.b).cuda()
    maxit = 4 * prob.n + 1000
    for _ in range(2):
        x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        st, k, _ = _noalloc(G, dims, b, x, 0.0, maxit)
        assert st in (G.PRCG_BREAKDOWN, G.PRCG_NOT_CONVERGED, G.PRCG_OK)
        assert (k == maxit) == (st == G.PRCG_NOT_CONVERGED) and k >= 1
        assert O.true_relres(A, prob.b, x.cpu().numpy()) <= 1e-13


def test_noalloc_allocates_nothing_and_rejects_large_n(G):
    import torch
    from paper_1905_01549_gb300 import binding
    prob = P.grid_problem((40, 30), "noalloc_mem", with_csr=False)
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    binding.prcg_pr_solve_stencil_noalloc(2, 40, 30, 1, 0.0, 0, b, x, 1e-10, 5000)  # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        x.zero_()
        status, _ = binding.prcg_pr_solve_stencil_noalloc(2, 40, 30, 1, 0.0, 0, b, x, 1e-10, 5000)
        assert status == G.PRCG_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    big = torch.zeros(65537, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.PrcgError):
        binding.prcg_pr_solve_stencil_noalloc(2, 65537, 1, 1, 0.0, 0, big, big.clone(), 1e-8, 10)
    # extents whose product would overflow 64 bits are refused before it is formed
    with pytest.raises(binding.PrcgError):
        binding.prcg_pr_solve_stencil_noalloc(3, 1 << 40, 1 << 40, 1 << 40, 0.0, 0, b, x, 1e-8, 10)
    # maxit above 4 n + 1000 is refused (the solve cannot be interrupted)
    with pytest.raises(binding.PrcgError):
        binding.prcg_pr_solve_stencil_noalloc(2, 40, 30, 1, 0.0, 0, b, x, 0.0, 4 * 1200 + 1001)
    # memory of another GPU is refused without a launch
    if torch.cuda.device_count() > 1:
        b1 = b.to("cuda:1")
        with pytest.raises(binding.PrcgError):
            binding.prcg_pr_solve_stencil_noalloc(2, 40, 30, 1, 0.0, 0, b1, x, 1e-8, 10)
    with pytest.raises(binding.PrcgError):   # host pointers are refused
        binding.prcg_pr_solve_stencil_noalloc(2, 40, 30, 1, 0.0, 0, prob.b, np.zeros(prob.n),
                                              1e-8, 10)
