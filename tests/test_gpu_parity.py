"""GPU (C ABI) vs CPU oracle, element by element on the same seeded inputs.

Bar (from the method's statement of the target): FP64 iterates within 1e-10
relative of the oracle over the first 20 iterations, the iteration count to
the tolerance within 5 %, and the final true residual at the tolerance.
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import CASES, GPU_VARIANTS, case, csr_matrix, make_solver, oracle_spread, rel

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10     # relative, first 20 iterations
HIST_TOL = 1e-9      # per entry of ||r_k|| / ||b||
SPREAD_FACTOR = 100.0


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


_KAPPA = {}


def _kappa(name):
    """Spectral condition number of a small parity case (dense eigenvalues)."""
    if name not in _KAPPA:
        ev = np.linalg.eigvalsh(csr_matrix(case(name)).toarray())
        _KAPPA[name] = float(ev[-1] / ev[0])
    return _KAPPA[name]


def _oracle_d(A, precond):
    return O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("op", ["csr", "stencil"])
@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_first_20_iterations(G, torch_mod, name, op, precond):
    torch = torch_mod
    prob = case(name)
    A = csr_matrix(prob)
    d = _oracle_d(A, precond)
    b = torch.from_numpy(prob.b).cuda()
    with make_solver(G, prob, op, precond) as S:
        for variant in GPU_VARIANTS:
            for k in (1, 2, 7, 20):
                res = S.solve(b, variant=variant, tol=0.0, maxit=k, history=True)
                ref, sx, sh = oracle_spread(variant, A, prob.b, d, k)
                assert res.status == ref.status == O.NOT_CONVERGED
                assert res.iters == k
                tol_x = max(ITER_TOL, SPREAD_FACTOR * sx)
                tol_h = max(HIST_TOL, SPREAD_FACTOR * sh)
                assert rel(res.x.cpu().numpy(), ref.x) <= tol_x, (variant, k, tol_x)
                h = np.asarray(ref.hist)
                assert np.all(np.abs(res.hist - h) <= tol_h * h), (variant, k, tol_h)
                if name in ("poisson2d_64", "poisson3d_ragged", "shifted2d") or precond == "jacobi":
                    assert tol_x == ITER_TOL  # well-conditioned: the plain 1e-10 bar


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("op", ["csr", "stencil"])
@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_converged_solve(G, torch_mod, name, op, precond):
    torch = torch_mod
    prob = case(name)
    A = csr_matrix(prob)
    d = _oracle_d(A, precond)
    b = torch.from_numpy(prob.b).cuda()
    tol = 1e-10
    with make_solver(G, prob, op, precond) as S:
        for variant in GPU_VARIANTS:
            ref = O.solve(variant, A, prob.b, d=d, tol=tol, maxit=4 * prob.n)
            res = S.solve(b, variant=variant, tol=tol, maxit=4 * prob.n, history=True,
                          true_relres=True)
            assert res.status == ref.status == O.OK, variant
            assert abs(res.iters - ref.iters) <= max(1, 0.05 * ref.iters), (variant, res.iters, ref.iters)
            assert res.hist[-1] <= tol
            assert res.true_relres <= 20 * tol, (variant, res.true_relres)
            # two solutions with true relative residuals t1, t2 differ by at
            # most kappa (t1 + t2) relative (the pre-conditioned kappa when
            # Jacobi is used is smaller; the unpreconditioned one bounds both)
            bound = 2 * _kappa(name) * (res.true_relres + O.true_relres(A, prob.b, ref.x))
            assert rel(res.x.cpu().numpy(), ref.x) <= max(1e-9, bound), (variant, bound)


def test_nonzero_x0_and_host_pointers(G, torch_mod):
    torch = torch_mod
    prob = case("poisson3d_ragged")
    A = csr_matrix(prob)
    x0 = np.random.default_rng(4).standard_normal(prob.n)
    with make_solver(G, prob, "csr", "jacobi") as S:
        for variant in GPU_VARIANTS:
            ref = O.solve(variant, A, prob.b, x0=x0.copy(), d=O.jacobi_inverse_diagonal(A),
                          tol=0.0, maxit=15)
            # host (numpy) b and x: the library copies in and out
            xh = x0.copy()
            res = S.solve(prob.b, x0=xh, variant=variant, tol=0.0, maxit=15)
            assert res.x is xh and rel(xh, ref.x) <= ITER_TOL
            # device tensors, x updated in place
            xd = torch.from_numpy(x0.copy()).cuda()
            res = S.solve(torch.from_numpy(prob.b).cuda(), x0=xd, variant=variant, tol=0.0, maxit=15)
            assert rel(xd.cpu().numpy(), ref.x) <= ITER_TOL


def test_edge_cases(G, torch_mod):
    torch = torch_mod
    prob = case("poisson2d_64")
    A = csr_matrix(prob)
    with make_solver(G, prob, "stencil", "none") as S:
        for variant in GPU_VARIANTS:
            # b = 0: x = 0, K = 0
            x = torch.ones(prob.n, dtype=torch.float64, device="cuda")
            res = S.solve(torch.zeros_like(x), x0=x, variant=variant, tol=1e-10, maxit=100)
            assert res.status == G.PRCG_OK and res.iters == 0 and float(x.abs().max()) == 0.0
            # x0 = exact solution of a system built from it: K = 0 at tol 1e-12
            xt = torch.from_numpy(prob.x_true).cuda()
            res = S.solve(torch.from_numpy(prob.b).cuda(), x0=xt.clone(), variant=variant,
                          tol=1e-12, maxit=100, history=True)
            assert res.iters == 0 and res.status == G.PRCG_OK
            # maxit = 0 and a tiny maxit
            res = S.solve(torch.from_numpy(prob.b).cuda(), variant=variant, tol=1e-10, maxit=0)
            assert res.status == G.PRCG_NOT_CONVERGED and res.iters == 0
            res = S.solve(torch.from_numpy(prob.b).cuda(), variant=variant, tol=1e-10, maxit=3)
            assert res.status == G.PRCG_NOT_CONVERGED and res.iters == 3


def test_n_equals_one_and_one_tile(G, torch_mod):
    torch = torch_mod
    import problems as P
    for dims in [(1, 1), (16, 16), (1, 1, 1), (256, 1), (257, 1)]:
        prob = P.grid_problem(dims, "t_small")
        A = csr_matrix(prob)
        for op in ("csr", "stencil"):
            with make_solver(G, prob, op, "jacobi") as S:
                for variant in GPU_VARIANTS:
                    ref = O.solve(variant, A, prob.b, d=O.jacobi_inverse_diagonal(A), tol=1e-12,
                                  maxit=4 * prob.n + 4)
                    res = S.solve(torch.from_numpy(prob.b).cuda(), variant=variant, tol=1e-12,
                                  maxit=4 * prob.n + 4)
                    assert res.status == ref.status and abs(res.iters - ref.iters) <= 1, (dims, op, variant)
                    assert rel(res.x.cpu().numpy(), ref.x) <= 1e-9


def test_breakdown_on_indefinite_matrix(G, torch_mod):
    """An indefinite symmetric A: the oracle and the GPU stop with BREAKDOWN at
    the same iteration (mu <= 0 or nu' < 0, Section 3.1)."""
    torch = torch_mod
    import scipy.sparse as sp
    n = 300
    rng = np.random.default_rng(8)
    diag = rng.uniform(1.0, 2.0, n)
    diag[::7] *= -1.0
    A = sp.diags([np.full(n - 1, 0.3), diag, np.full(n - 1, 0.3)], [-1, 0, 1], format="csr")
    b = rng.standard_normal(n)
    with G.Solver.from_csr(A.indptr, A.indices, A.data) as S:
        for variant in GPU_VARIANTS:
            ref = O.solve(variant, A, b, tol=1e-12, maxit=2000)
            res = S.solve(torch.from_numpy(b).cuda(), variant=variant, tol=1e-12, maxit=2000)
            assert ref.status == O.BREAKDOWN
            assert res.status == G.PRCG_BREAKDOWN and res.iters == ref.iters, (variant, res.iters, ref.iters)


def test_invalid_inputs_are_rejected(G):
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([0, 5], dtype=np.int32)        # column out of range
    v = np.array([1.0, 1.0])
    with pytest.raises(G.PrcgError):
        G.Solver.from_csr(rp, ci, v)
    ci = np.array([1, 0], dtype=np.int32)        # no diagonal: Jacobi impossible
    with pytest.raises(G.PrcgError):
        G.Solver.from_csr(rp, ci, v, precond="jacobi")
    rp_bad = np.array([0, 2, 1], dtype=np.int32)  # decreasing row_ptr
    with pytest.raises(G.PrcgError):
        G.Solver.from_csr(rp_bad, np.array([0, 1], dtype=np.int32), v)
    S = G.Solver.from_stencil((8, 8))
    with pytest.raises(G.PrcgError):
        S.solve(np.ones(64), variant="pr", tol=-1.0)
    with pytest.raises(G.PrcgError):
        S.solve(np.ones(64), variant="pr", tol=1e-8, maxit=-1)
    S.close()


def test_reruns_are_bitwise_identical(G, torch_mod):
    """Fixed-order reductions: the same solve twice gives identical bits."""
    torch = torch_mod
    prob = case("varcoef3d_ragged")
    b = torch.from_numpy(prob.b).cuda()
    with make_solver(G, prob, "csr", "jacobi") as S:
        for variant in GPU_VARIANTS:
            r1 = S.solve(b, variant=variant, tol=1e-10, maxit=5000, history=True)
            r2 = S.solve(b, variant=variant, tol=1e-10, maxit=5000, history=True)
            assert r1.iters == r2.iters
            assert torch.equal(r1.x, r2.x) and np.array_equal(r1.hist, r2.hist)


@pytest.mark.parametrize("name,op,precond", [("poisson3d_ragged", "csr", "jacobi"),
                                             ("varcoef2d_ragged", "csr", "jacobi"),
                                             ("varcoef3d_ragged", "stencil", "jacobi"),
                                             ("poisson2d_64", "stencil", "none")])
def test_persistent_and_graph_paths_match_oracle(G, torch_mod, name, op, precond, monkeypatch):
    """Small systems run as one persistent cooperative kernel by default; the
    graph path (PRCG_PERSIST_MAX=0) must give the same iterates."""
    torch = torch_mod
    prob = case(name)
    A = csr_matrix(prob)
    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
    b = torch.from_numpy(prob.b).cuda()
    xs = {}
    for mode in ("persistent", "graph"):
        if mode == "graph":
            monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
        with make_solver(G, prob, op, precond) as S:
            for variant in GPU_VARIANTS:
                res = S.solve(b, variant=variant, tol=0.0, maxit=20)
                ref = O.solve(variant, A, prob.b, d=d, tol=0.0, maxit=20)
                assert rel(res.x.cpu().numpy(), ref.x) <= ITER_TOL, (mode, variant)
                xs[(mode, variant)] = res.x.cpu().numpy()
                from paper_1905_01549_gb300 import binding
                launches = binding.prcg_last_launches(S.handle)
                assert (launches == 1) == (mode == "persistent"), (mode, launches)
        monkeypatch.delenv("PRCG_PERSIST_MAX", raising=False)


@pytest.mark.parametrize("path", ["persistent", "graph"])
def test_nan_in_b_reports_breakdown_and_context_recovers(G, torch_mod, path, monkeypatch):
    """Host-side fault injection: a NaN in b makes the first scalars
    non-finite; every variant stops with BREAKDOWN after initialize() (as the
    oracle does), nothing hangs, and the context then solves normally."""
    torch = torch_mod
    if path == "graph":
        monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = case("poisson3d_ragged")
    A = csr_matrix(prob)
    bad = prob.b.copy()
    bad[prob.n // 2] = np.nan
    with make_solver(G, prob, "stencil", "jacobi") as S:
        for variant in GPU_VARIANTS:
            ref = O.solve(variant, A, bad, d=O.jacobi_inverse_diagonal(A), tol=1e-10, maxit=50)
            res = S.solve(torch.from_numpy(bad).cuda(), variant=variant, tol=1e-10, maxit=50)
            assert ref.status == O.BREAKDOWN
            assert res.status == G.PRCG_BREAKDOWN and res.iters == ref.iters == 0, variant
        res = S.solve(torch.from_numpy(prob.b).cuda(), variant="pr", tol=1e-10, maxit=1000)
        assert res.status == G.PRCG_OK


@pytest.mark.parametrize("path", ["persistent", "graph"])
@pytest.mark.parametrize("name", ["poisson3d_ragged", "shifted2d"])
def test_point_source_mixes_fallback_and_fixed_point_rows(G, torch_mod, name, path, monkeypatch):
    """b = a point source: for the first iterations most rows of p see only
    exact zeros (the stencil's neighbour sum then takes its FP64 fallback)
    next to rows in the fixed-point window; the iterates still match the
    oracle element by element."""
    torch = torch_mod
    if path == "graph":
        monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = case(name)
    A = csr_matrix(prob)
    b = np.zeros(prob.n)
    b[prob.n // 3] = 1.0
    with make_solver(G, prob, "stencil", "none") as S:
        for variant in ("hs", "pr", "pipe_pr"):
            for k in (1, 3, 8, 20):
                res = S.solve(torch.from_numpy(b).cuda(), variant=variant, tol=0.0, maxit=k,
                              history=True)
                ref, sx, sh = oracle_spread(variant, A, b, None, k)
                assert res.iters == ref.iters == k, (variant, k)
                tol_x = max(ITER_TOL, SPREAD_FACTOR * sx)
                assert rel(res.x.cpu().numpy(), ref.x) <= tol_x, (variant, k, tol_x)


@pytest.mark.parametrize("path", ["persistent", "graph"])
def test_exact_initial_guess_stops_at_zero_iterations(G, torch_mod, path, monkeypatch):
    """x_0 = A^{-1} b exactly (integer x_0, integer stencil, so b = A x_0 and
    r_0 = 0 in floating point): every variant returns OK with K = 0 and x_0."""
    torch = torch_mod
    if path == "graph":
        monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    import problems as P
    dims = (13, 9, 7)
    x0 = np.random.default_rng(4).integers(-5, 6, 13 * 9 * 7).astype(np.float64)
    b = P.stencil_apply(dims, x0)          # integers: exact, so r_0 = b - A x_0 = 0
    with G.Solver.from_stencil(dims) as S:
        for variant in GPU_VARIANTS:
            x = torch.from_numpy(x0.copy()).cuda()
            res = S.solve(torch.from_numpy(b).cuda(), x0=x, variant=variant, tol=1e-12, maxit=100,
                          history=True)
            assert res.status == G.PRCG_OK and res.iters == 0, variant
            assert np.array_equal(x.cpu().numpy(), x0) and res.hist[0] == 0.0


def test_graph_path_reruns_are_bitwise_identical(G, torch_mod, monkeypatch):
    torch = torch_mod
    monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = case("varcoef3d_ragged")
    b = torch.from_numpy(prob.b).cuda()
    with make_solver(G, prob, "csr", "jacobi") as S:
        for variant in GPU_VARIANTS:
            r1 = S.solve(b, variant=variant, tol=1e-10, maxit=5000, history=True)
            r2 = S.solve(b, variant=variant, tol=1e-10, maxit=5000, history=True)
            assert r1.iters == r2.iters
            assert torch.equal(r1.x, r2.x) and np.array_equal(r1.hist, r2.hist)
