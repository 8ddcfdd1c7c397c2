"""The allocation-free PR-CG entry point against the regular one.

prcg_pr_solve_stencil_noalloc exists for callers that cannot allocate
device memory (foreign memory pools, real-time loops without cudaMalloc);
it keeps its iteration vectors in a fixed file-scope device array.  Here it
is called through the C ABI twice in a row (the second call must not see the
first call's leftovers) and compared with prcg_solve on the same inputs.
This file sorts last so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import problems as P
from gpu_common import rel

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
    finally:
        regular.close()


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
    with pytest.raises(binding.PrcgError):   # host pointers are refused
        binding.prcg_pr_solve_stencil_noalloc(2, 40, 30, 1, 0.0, 0, prob.b, np.zeros(prob.n),
                                              1e-8, 10)
