"""Dense-matrix path (Section 5's dense model problem) against the oracle.

Every product with a dense A is formed by a column-block pre-pass; the
variants then run unchanged.  The bars are the parity tests' bars: FP64
iterates within 1e-10 of the oracle over the first 20 iterations, the
iteration count to the tolerance within 5 %, the final true residual at the
tolerance -- on the persistent path and on the graph path.
"""
import numpy as np
import pytest

import oracle as O
import problems as P
from gpu_common import GPU_VARIANTS, ITER_TOL, OracleBand, rel

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


def _cases():
    # rho = 1 in Eq. 4.1 spaces the spectrum evenly over [0.1, 1] (kappa 10):
    # the iterates are insensitive to rounding, so the 1e-10 bar applies as is.
    # The clustered Eq. 4.1 spectra (rho < 1) make the iterates themselves
    # sensitive to summation order; there the bar is 8 x the oracle's own
    # spread over three other roundings, never above 1e-6, as in the
    # sparse parity tests.
    return {
        "uniform_96": (P.model_problem(96, 1.0, 10.0), "none"),
        "uniform_77_jacobi": (P.model_problem(77, 1.0, 10.0), "jacobi"),
        "model_200": (P.model_problem(200, 0.9, 1e3), "none"),
        "model_77_jacobi": (P.model_problem(77, 0.8, 1e2), "jacobi"),
        "one": (P.DenseProblem(np.array([[4.0]]), np.array([2.0]), np.array([0.5]), np.empty(0)),
                "jacobi"),
    }


CASES = _cases()


@pytest.mark.parametrize("path", ["persistent", "graph"])
@pytest.mark.parametrize("name", list(CASES))
def test_dense_first_20_iterations(G, name, path, monkeypatch):
    import torch
    prob, pc = CASES[name]
    if path == "graph":
        monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    d = O.jacobi_inverse_diagonal(prob.A) if pc == "jacobi" else None
    b = torch.from_numpy(prob.b).cuda()
    with G.Solver.from_dense(prob.A, precond=pc) as S:
        for v in GPU_VARIANTS:
            k = min(20, len(prob.b))
            res = S.solve(b, variant=v, tol=0.0, maxit=k)
            band = OracleBand(v, prob.A, prob.b, d, k)
            if name.startswith("uniform"):
                assert band.bar_x(k) == ITER_TOL, (v, band.spread_x(k))
            assert res.iters == band.ref.iters, (v, res.iters, band.ref.iters)
            # the first k' <= k iterations where x is determined to 1e-6
            kd = max(j for j in range(k + 1) if band.determined(j))
            assert kd >= min(k, 10), (v, kd)
            if kd < k:
                res = S.solve(b, variant=v, tol=0.0, maxit=kd)
            xg = res.x.cpu().numpy()
            assert band.dist_x(kd, xg) <= band.bar_x(kd), (v, kd, band.dist_x(kd, xg),
                                                          band.bar_x(kd))
            from paper_1905_01549_gb300 import binding
            launches = binding.prcg_last_launches(S.handle)
            persistent = path == "persistent"
            assert (launches == 1) == persistent, (v, launches)


@pytest.mark.parametrize("variant", GPU_VARIANTS)
def test_dense_converged_solve(G, variant):
    import torch
    prob, _ = CASES["model_200"]
    b = torch.from_numpy(prob.b).cuda()
    tol = 1e-8 if variant == "gv" else 1e-10
    with G.Solver.from_dense(torch.from_numpy(prob.A).cuda()) as S:
        res = S.solve(b, variant=variant, tol=tol, maxit=4000, true_relres=True)
    ref = O.solve(variant, prob.A, prob.b, tol=tol, maxit=4000)
    # the oracle with exactly rounded inner products: on this clustered
    # spectrum GV-CG's count moves by ~5 % under summation order alone
    import math
    import oracle.cg_variants as CV
    saved = CV._dot
    CV._dot = lambda u, v: saved(u, v) if u.dtype == object else math.fsum(u * v)
    try:
        alt = O.solve(variant, prob.A, prob.b, tol=tol, maxit=4000)
    finally:
        CV._dot = saved
    assert res.status == 0 and ref.status == 0
    bar = max(1, 0.05 * ref.iters, 2 * abs(alt.iters - ref.iters))
    assert abs(res.iters - ref.iters) <= bar, (res.iters, ref.iters, alt.iters)
    assert res.true_relres <= 10 * tol


def test_dense_reruns_bitwise_and_host_arrays(G):
    import torch
    prob, pc = CASES["uniform_77_jacobi"]
    with G.Solver.from_dense(prob.A, precond=pc) as S:
        r1 = S.solve(prob.b, x0=np.zeros(77), variant="pipe_pr", tol=1e-12, maxit=500, history=True)
        r2 = S.solve(torch.from_numpy(prob.b).cuda(), variant="pipe_pr", tol=1e-12, maxit=500,
                     history=True)
    assert r1.iters == r2.iters and np.array_equal(r1.hist, r2.hist)
    assert np.array_equal(r1.x, r2.x.cpu().numpy())


def test_dense_errors(G):
    A = np.array([[1.0, 2.0], [2.0, -1.0]])
    with pytest.raises(G.PrcgError) as e:
        G.Solver.from_dense(A, precond="jacobi")
    assert e.value.code == -1
    prob, _ = CASES["uniform_77_jacobi"]
    with G.Solver.from_dense(prob.A) as S:
        with pytest.raises(G.PrcgError) as e:
            S.solve_refined_fp32(prob.b)
        assert e.value.code == -5


def test_dense_full_size_first_iterations(G):
    """Section 5's size, n = 10752 (A = 925 MB, 29 column blocks on 152 SMs),
    in the launch configuration the bench times; a dense SPD matrix built in
    O(n^2) stands in for the model problem (whose host QR takes minutes)."""
    import torch
    n = 10752
    prob = P.dense_lowrank_spd(n, 8, P.rng_for("dense10752"))
    d = O.jacobi_inverse_diagonal(prob.A)
    b = torch.from_numpy(prob.b).cuda()
    with G.Solver.from_dense(prob.A, precond="jacobi") as S:
        for v in ("hs", "pr", "pipe_pr"):
            res = S.solve(b, variant=v, tol=0.0, maxit=3)
            ref = O.solve(v, prob.A, prob.b, d=d, tol=0.0, maxit=3)
            assert rel(res.x.cpu().numpy(), ref.x) <= ITER_TOL, v
