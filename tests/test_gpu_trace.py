"""The scalars of every iteration (prcg_trace_*) against the oracle's.

The parity bar covers the scalars as well as the vectors: alpha, beta, nu,
nu', mu, sigma, gamma, rho and eta of the first 20 iterations must match
the oracle's to 1e-10 relative -- or, where the iterates themselves are
sensitive to summation order, to 100 x the oracle's own spread under
exactly rounded inner products (the rule of the vector parity tests).  The
trace also lets the GPU be checked against Section 3.1's bound on the gap
between the predicted nu'_k and the recomputed <r_k, r_k>.
"""
import math

import numpy as np
import pytest

import oracle as O
import problems as P
from gpu_common import GPU_VARIANTS, case, csr_matrix, make_solver

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10
SPREAD_FACTOR = 100.0
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


def _oracle_scalars(variant, A, b, d, k, exact_dots=False):
    import oracle.cg_variants as CV
    saved = CV._dot
    if exact_dots:
        CV._dot = lambda u, v: saved(u, v) if u.dtype == object else math.fsum(u * v)
    try:
        return O.solve(variant, A, b, d=d, tol=0.0, maxit=k)
    finally:
        CV._dot = saved


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _compare(tr, ref, alt):
    """Worst relative difference GPU vs oracle, and the oracle's own spread,
    over every scalar the oracle formed."""
    worst, spread = 0.0, 0.0
    last = len(ref.scalars) - 1
    for k, sc in enumerate(ref.scalars):
        for f, v in sc.items():
            g = tr[k, FIELDS.index(f)]
            if k == last and f in ("beta", "mu") and not np.isfinite(g):
                continue   # formed by the oracle after its final stopping test, never used
            assert np.isfinite(g), (k, f)
            worst = max(worst, _rel(g, v))
            spread = max(spread, _rel(alt.scalars[k][f], v))
    return worst, spread


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
            ref = _oracle_scalars(v, A, prob.b, d, k)
            alt = _oracle_scalars(v, A, prob.b, d, k, exact_dots=True)
            assert res.iters == ref.iters == k
            assert res.trace.shape == (k + 1, 10)
            worst, spread = _compare(res.trace, ref, alt)
            assert worst <= max(ITER_TOL, SPREAD_FACTOR * spread), (v, worst, spread)


def test_trace_off_by_default_and_dense(G):
    import torch
    prob = P.model_problem(96, 1.0, 10.0)
    b = torch.from_numpy(prob.b).cuda()
    with G.Solver.from_dense(prob.A) as S:
        assert S.solve(b, variant="pr", tol=0.0, maxit=5).trace is None
        res = S.solve(b, variant="pipe_pr", tol=0.0, maxit=15, trace=True)
    ref = O.solve("pipe_pr", prob.A, prob.b, tol=0.0, maxit=15)
    alt = _oracle_scalars("pipe_pr", prob.A, prob.b, None, 15, exact_dots=True)
    worst, spread = _compare(res.trace, ref, alt)
    assert worst <= max(ITER_TOL, SPREAD_FACTOR * spread), (worst, spread)


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
