"""Convergence study on the GPU (Section 4, Table 2) against the oracle.

The statistics of Table 2 -- iterations to a 10^5 reduction of the A-norm
error and the minimum error reached -- computed from the GPU variants'
iterates must agree with the same statistics of the oracle's iterates on the
same seeded model problem, and the paper's accuracy ordering (GV-CG loses
orders of magnitude, pipe-PR-CG stays near HS-CG) must hold on the GPU.
"""
import math

import numpy as np
import pytest

import oracle as O
import problems as P
from gpu_common import GPU_VARIANTS, rel

pytestmark = pytest.mark.gpu

KMAX = 200


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


def _dense_csr(A):
    n = A.shape[0]
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    return rp, ci, np.ascontiguousarray(A.ravel())


def _oracle_stats(variant, prob, d, exact_dots=False):
    """Table 2's statistics of the oracle's iterates; with exact_dots the inner
    products are exactly rounded (math.fsum) instead of numpy's order."""
    import oracle.cg_variants as CV
    saved = CV._dot
    if exact_dots:
        CV._dot = lambda u, v: saved(u, v) if u.dtype == object else math.fsum(u * v)
    try:
        res = O.solve(variant, prob.A, prob.b, d=d, maxit=KMAX, record=KMAX)
    finally:
        CV._dot = saved
    e0 = O.a_norm_error(prob.A, prob.x_star, np.zeros_like(prob.b))
    errs = np.array([O.a_norm_error(prob.A, prob.x_star, x) / e0 for x, _ in res.iterates])
    hit = np.nonzero(errs <= 1e-5)[0]
    return (int(hit[0]) if len(hit) else None), math.log10(errs.min())


@pytest.fixture(scope="module")
def model():
    return P.model_problem(48, 0.8, 1e3)


def test_error_anorm_matches_oracle(G, model):
    import torch
    rp, ci, v = _dense_csr(model.A)
    rng = np.random.default_rng(3)
    x = model.x_star + 1e-3 * rng.standard_normal(48)
    with G.Solver.from_csr(rp, ci, v) as S:
        got = S.error_anorm(torch.from_numpy(model.x_star).cuda(), torch.from_numpy(x).cuda())
        got_host = S.error_anorm(model.x_star, x)
    ref = O.a_norm_error(model.A, model.x_star, x)
    assert abs(got - ref) <= 1e-12 * ref and got == got_host


@pytest.mark.parametrize("precond", ["none", "jacobi"])
@pytest.mark.parametrize("variant", GPU_VARIANTS)
def test_table2_statistics_match_oracle(G, model, variant, precond):
    import torch
    from paper_1905_01549_gb300 import convergence
    d = O.jacobi_inverse_diagonal(model.A) if precond == "jacobi" else None
    rp, ci, v = _dense_csr(model.A)
    with G.Solver.from_csr(rp, ci, v, precond=precond) as S:
        curve = convergence.error_curve(S, torch.from_numpy(model.b).cuda(),
                                        torch.from_numpy(model.x_star).cuda(), variant, KMAX)
    k5, emin = curve.iterations_to(1e5), curve.min_log10()
    ok5, oemin = _oracle_stats(variant, model, d)
    # The error curve has plateaus near 1e-5 on this spectrum, so the crossing
    # index moves with summation order alone: the oracle with exactly rounded
    # inner products crosses up to 2 iterations away from the plain oracle.
    # Bar: 2 iterations plus that spread on this case.
    sk5, _ = _oracle_stats(variant, model, d, exact_dots=True)
    assert k5 is not None and abs(k5 - ok5) <= 2 + abs(sk5 - ok5), (k5, ok5, sk5)
    # GV-CG's attainable accuracy is set by rounding errors that its auxiliary
    # recurrences amplify (the reason Table 2 shows it 4 decades behind HS), so
    # its level moves by a factor of a few between FP64 implementations that
    # round differently (FMA contraction on the GPU, none in the oracle).
    assert abs(emin - oemin) <= (1.0 if variant == "gv" else 0.5), (emin, oemin)
    # the curves agree closely while rounding is negligible (first 10 iterations)
    res = O.solve(variant, model.A, model.b, d=d, maxit=10, record=10)
    e0 = O.a_norm_error(model.A, model.x_star, np.zeros(48))
    oerrs = np.array([O.a_norm_error(model.A, model.x_star, x) / e0 for x, _ in res.iterates])
    assert rel(curve.err[:11], oerrs) <= 1e-9


def test_accuracy_ordering_on_gpu(G, model):
    """Table 2's central observation on the GPU: GV-CG's attainable accuracy is
    orders of magnitude worse than HS-CG's, pipe-PR-CG's within a decade."""
    import torch
    from paper_1905_01549_gb300 import convergence
    rp, ci, v = _dense_csr(model.A)
    with G.Solver.from_csr(rp, ci, v) as S:
        st = convergence.study(S, torch.from_numpy(model.b).cuda(),
                               torch.from_numpy(model.x_star).cuda(), ["hs", "pipe_pr", "gv"], KMAX)
    e_hs, e_ppr, e_gv = (st[v]["min_log10_err"] for v in ("hs", "pipe_pr", "gv"))
    assert e_gv > e_hs + 3, st
    assert e_ppr < e_hs + 1, st
