"""prcg_time_sweeps: the per-sweep timer that the benchmark's rooflines use.

It runs initialize() and `reps` iterations with the stopping tests off on
the context's own vectors.  Checked here: the number of sweeps each variant
reports (HS 3, PR / M / CG-CG 2, pipe-PR / pipe-M / GV 1), positive finite
times, the ablations refused, and that a solve after the timing run still
matches the oracle (Algorithms 1-3), i.e. the timer leaves nothing behind
that a later solve reads.
"""
import math

import numpy as np
import pytest

import oracle as O
import problems as P
from gpu_common import csr_matrix, rel

pytestmark = pytest.mark.gpu

SWEEPS = {"hs": 3, "pr": 2, "m": 2, "cgcg": 2, "pipe_pr": 1, "pipe_m": 1, "gv": 1}


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


@pytest.mark.parametrize("op", ["stencil", "csr"])
@pytest.mark.parametrize("precond", ["none", "jacobi"])
@pytest.mark.parametrize("persist_max", [None, "0"])
def test_time_sweeps_then_solve(G, op, precond, persist_max, monkeypatch):
    import torch
    from paper_1905_01549_gb300 import binding
    if persist_max is not None:
        monkeypatch.setenv("PRCG_PERSIST_MAX", persist_max)
    prob = P.grid_problem((24, 20, 18), "timing")
    A = csr_matrix(prob)
    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
    if op == "stencil":
        S = G.Solver.from_stencil(prob.dims, precond=precond)
    else:
        S = G.Solver.from_csr(A.indptr.astype(np.int32), A.indices.astype(np.int32),
                              A.data.astype(np.float64), precond=precond)
    b = torch.from_numpy(prob.b).cuda()
    with S:
        for v, k in SWEEPS.items():
            ms = binding.prcg_time_sweeps(S.handle, binding.VARIANT_IDS[v], 5)
            assert len(ms) == k, (v, ms)
            assert all(math.isfinite(t) and t > 0.0 for t in ms), (v, ms)
        for v in ("pr_norecompute", "pipe_pr_norecompute"):
            with pytest.raises(binding.PrcgError):
                binding.prcg_time_sweeps(S.handle, binding.VARIANT_IDS[v], 5)
        for v in ("hs", "pr", "pipe_pr"):
            binding.prcg_time_sweeps(S.handle, binding.VARIANT_IDS[v], 7)
            ref = O.solve(v, A, prob.b, d=d, tol=1e-10, maxit=2000)
            res = S.solve(b, variant=v, tol=1e-10, maxit=2000)
            assert res.status == ref.status == O.OK
            assert abs(res.iters - ref.iters) <= 1, (v, res.iters, ref.iters)
            assert rel(res.x.cpu().numpy(), ref.x) <= 1e-8
