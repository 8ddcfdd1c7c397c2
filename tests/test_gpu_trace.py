"""The scalars of every iteration (prcg_trace_*) against the oracle's.

The parity bar covers the scalars as well as the vectors: alpha, beta, nu,
nu', mu, sigma, gamma, rho and eta of the first 20 iterations must match
the oracle's to 1e-10 relative -- or, where the iterates themselves are
sensitive to summation order, to 8 x the oracle's own spread over three other
rounding orders, never above 1e-6 (the rule of the vector parity tests,
gpu_common.OracleBand).  The trace also lets the GPU be checked against
Section 3.1's bound on the gap between the predicted nu'_k and the
recomputed <r_k, r_k>.
"""
import numpy as np
import pytest

import oracle as O
import problems as P
from gpu_common import (DETERMINED, GPU_VARIANTS, ITER_TOL, SPREAD_FACTOR, OracleBand, case,
                        csr_matrix, make_solver)

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53
FIELDS = ("alpha", "beta", "nu", "nu_pred", "mu", "sigma", "gamma", "rho", "eta")


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _compare(tr, band):
    """Worst ratio of the GPU's distance to the nearest oracle run over the
    bar, over every scalar the oracle formed in the iterations where the
    scalars are determined (the bar, 8 x the spread of the oracle runs
    growing with k, stays within DETERMINED); returns (worst, compared)."""
    ref = band.ref
    last = len(ref.scalars) - 1
    spread, worst, compared = 0.0, 0.0, 0
    for k, sc in enumerate(ref.scalars):
        spread = max([spread, band.spread_x(k)] +
                     [_rel(a.scalars[k][f], v) for a in band.alts for f, v in sc.items()])
        bar = max(ITER_TOL, SPREAD_FACTOR * spread)
        for f, v in sc.items():
            g = tr[k, FIELDS.index(f)]
            if k == last and f in ("beta", "mu") and not np.isfinite(g):
                continue   # formed by the oracle after its final stopping test, never used
            assert np.isfinite(g), (k, f)
            if bar > DETERMINED:
                continue
            dist = min(_rel(g, r.scalars[k][f]) for r in band.runs)
            worst = max(worst, dist / bar)
            compared += 1
    return worst, compared


@pytest.mark.parametrize("path", ["persistent", "graph"])
@pytest.mark.parametrize("name,op,precond", [("poisson3d_ragged", "csr", "jacobi"),
                                             ("varcoef2d_ragged", "stencil", "none"),
                                             ("poisson2d_64", "stencil", "jacobi")])
def test_scalar_trace_matches_oracle(G, name, op, precond, path, monkeypatch):
    import torch
    if path == "graph":
        monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = case(name)
    A = csr_matrix(prob)
    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
    b = torch.from_numpy(prob.b).cuda()
    k = 20
    with make_solver(G, prob, op, precond) as S:
        for v in GPU_VARIANTS:
            res = S.solve(b, variant=v, tol=0.0, maxit=k, trace=True)
            band = OracleBand(v, A, prob.b, d, k)
            assert res.iters == band.ref.iters == k
            assert res.trace.shape == (k + 1, 10)
            worst, compared = _compare(res.trace, band)
            assert worst <= 1.0, (v, worst)
            # at least the first 15 iterations' scalars are compared everywhere
            assert compared >= 15 * 2, (v, compared)


def test_trace_off_by_default_and_dense(G):
    import torch
    prob = P.model_problem(96, 1.0, 10.0)
    b = torch.from_numpy(prob.b).cuda()
    with G.Solver.from_dense(prob.A) as S:
        assert S.solve(b, variant="pr", tol=0.0, maxit=5).trace is None
        res = S.solve(b, variant="pipe_pr", tol=0.0, maxit=15, trace=True)
    band = OracleBand("pipe_pr", prob.A, prob.b, None, 15)
    worst, compared = _compare(res.trace, band)
    assert worst <= 1.0 and compared > 15 * 4, (worst, compared)


def _nu_gap_worst(tr, n):
    """max_k |rho_k - nu'_k| / (eps (30 + 7n)(rho_{k-1} + rho_k)) over the trace."""
    rho = tr[:, FIELDS.index("rho")]
    nup = tr[:, FIELDS.index("nu_pred")]
    worst = 0.0
    for k in range(1, len(tr)):
        if not np.isfinite(rho[k]):
            break
        bound = EPS * (30 + 7 * n) * (rho[k - 1] + rho[k])
        worst = max(worst, abs(rho[k] - nup[k]) / bound)
    return worst


@pytest.mark.parametrize("path", ["persistent", "graph"])
@pytest.mark.parametrize("variant", ["pr", "pipe_pr"])
def test_nu_prime_gap_bound_on_gpu(G, variant, path, monkeypatch):
    """Section 3.1 (Eq. 3.16) on the GPU's own iterates: the predicted nu'_k
    differs from the recomputed <r_k, r_k> only by local rounding errors,
    also long after convergence (150 and 200 iterations)."""
    import torch
    if path == "graph":
        monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = P.model_problem(48, 0.8, 1e3)
    with G.Solver.from_dense(prob.A) as S:
        res = S.solve(torch.from_numpy(prob.b).cuda(), variant=variant, tol=0.0, maxit=150,
                      trace=True)
    assert res.iters == 150
    assert _nu_gap_worst(res.trace, 48) <= 1.0
    rng = np.random.default_rng(9)
    b = rng.uniform(-1, 1, 256)
    with G.Solver.from_stencil((16, 16)) as S:
        res = S.solve(torch.from_numpy(b).cuda(), variant=variant, tol=0.0, maxit=200, trace=True)
    assert res.iters == 200
    assert _nu_gap_worst(res.trace, 256) <= 1.0
