"""GPU (C ABI) vs CPU oracle, element by element on the same seeded inputs.

Bar (from the method's statement of the target): FP64 iterates within 1e-10
relative of the oracle over the first 20 iterations, the iteration count to
the tolerance within 5 %, and the final true residual at the tolerance.
Where a system makes the iterates themselves sensitive to rounding order,
the bar is 8 x the oracle's own spread over three other roundings,
never above 1e-6 (gpu_common.OracleBand); past that point properties are
checked instead.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
from gpu_common import (CASES, GPU_VARIANTS, ITER_TOL, OracleBand, case,
                        csr_matrix, make_solver, rel)

pytestmark = pytest.mark.gpu

HIST_TOL = 1e-9      # per entry of ||r_k|| / ||b||
KS = (1, 2, 7, 10, 15, 20)


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


def _well_conditioned(name, precond):
    return name in ("poisson2d_64", "poisson3d_ragged", "shifted2d") or precond == "jacobi"


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("op", ["csr", "stencil"])
@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_first_20_iterations(G, torch_mod, name, op, precond):
    torch = torch_mod
    prob = case(name)
    A = csr_matrix(prob)
    d = _oracle_d(A, precond)
    b = torch.from_numpy(prob.b).cuda()
    xstar = None
    with make_solver(G, prob, op, precond) as S:
        for variant in GPU_VARIANTS:
            band = OracleBand(variant, A, prob.b, d, KS[-1])
            prev_ea = None
            for k in KS:
                res = S.solve(b, variant=variant, tol=0.0, maxit=k, history=True)
                assert res.status == O.NOT_CONVERGED and res.iters == k
                xg = res.x.cpu().numpy()
                ok_h, worst_h = band.hist_ok(k, res.hist, HIST_TOL)
                assert ok_h, (variant, k, worst_h)
                if _well_conditioned(name, precond):
                    assert band.bar_x(k) == ITER_TOL, (variant, k, band.spread_x(k))
                if not _well_conditioned(name, precond):
                    # CG minimises the A-norm error: it decreases from one
                    # checkpoint to the next on the GPU's own iterates
                    if xstar is None:
                        xstar = spla.spsolve(A.tocsc(), prob.b)
                    ea = O.a_norm_error(A, xstar, xg)
                    if prev_ea is not None:
                        assert ea <= prev_ea, (variant, k)
                    prev_ea = ea
                if band.determined(k):
                    assert band.dist_x(k, xg) <= band.bar_x(k), (variant, k, band.dist_x(k, xg),
                                                                 band.bar_x(k))
                    continue
                # x_k is not determined to DETERMINED by FP64 arithmetic (an
                # unpreconditioned sigma = 2 diffusion case near k = 20): its
                # A-norm error, which CG minimises, lies within the oracle
                # runs' own spread (up to 7 % among themselves on these
                # cases), doubled, of the nearest run, and within 1 %
                # where they agree more closely
                assert k >= 15, (variant, k, band.spread_x(k))
                eas = [O.a_norm_error(A, xstar, r.iterates[k][0]) for r in band.runs]
                bar_ea = max(1e-2, 2.0 * (max(eas) - min(eas)) / min(eas))
                assert min(abs(ea - e) / e for e in eas) <= bar_ea, (variant, k, ea, eas)


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
                band = OracleBand(variant, A, b, None, k)
                assert res.iters == band.ref.iters == k, (variant, k)
                assert band.determined(k), (variant, k, band.spread_x(k))
                xg = res.x.cpu().numpy()
                assert band.dist_x(k, xg) <= band.bar_x(k), (variant, k, band.bar_x(k))


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


@pytest.mark.parametrize("path", ["persistent", "graph"])
def test_constant_csr_diagonal_runs_as_scalar(G, torch_mod, path, monkeypatch):
    """A CSR matrix whose diagonal is one constant (Poisson) applies Jacobi as
    a scalar; forced back to the d vector (PRCG_NO_SCALAR_D=1) the iterates
    are the same to the parity bar, and both match the oracle.  A varying
    diagonal keeps the vector."""
    torch = torch_mod
    if path == "graph":
        monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = case("poisson3d_ragged")
    A = csr_matrix(prob)
    d = O.jacobi_inverse_diagonal(A)
    b = torch.from_numpy(prob.b).cuda()
    forms = {}
    xs = {}
    for env in ("0", "1"):
        monkeypatch.setenv("PRCG_NO_SCALAR_D", env)
        with make_solver(G, prob, "csr", "jacobi") as S:
            forms[env] = S.jacobi_form
            for variant in GPU_VARIANTS:
                res = S.solve(b, variant=variant, tol=0.0, maxit=20)
                xs[(env, variant)] = res.x.cpu().numpy()
    assert forms == {"0": "scalar", "1": "vector"}
    for variant in GPU_VARIANTS:
        ref = O.solve(variant, A, prob.b, d=d, tol=0.0, maxit=20)
        for env in ("0", "1"):
            assert rel(xs[(env, variant)], ref.x) <= ITER_TOL, (variant, env)
    monkeypatch.setenv("PRCG_NO_SCALAR_D", "0")
    with make_solver(G, case("varcoef3d_ragged"), "csr", "jacobi") as S:
        assert S.jacobi_form == "vector"
    with make_solver(G, prob, "csr", "none") as S:
        assert S.jacobi_form == "none"


@pytest.mark.parametrize("path", ["persistent", "graph"])
@pytest.mark.parametrize("dims", [(20, 11, 7), (44, 31)])
@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_two_row_face_stencil_matches_csr_and_oracle(G, torch_mod, path, dims, precond,
                                                     monkeypatch):
    """With an even nx the face-coefficient stencil forms two rows of a grid
    line per thread (one load of the shared x-face, 16-byte loads of the
    rest).  Each row's FMA chain is the CSR row's, in the same column order
    with the same coefficients; only the order in which a thread adds its
    rows into the inner products changes.  So the face stencil and the same
    matrix as CSR agree to rounding level over the first iterations, and the
    face stencil matches the oracle under the parity bar."""
    torch = torch_mod
    if path == "graph":
        monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    import problems as P
    prob = P.grid_problem(dims, "t_pair", sigma=2.0)
    A = csr_matrix(prob)
    d = _oracle_d(A, precond)
    b = torch.from_numpy(prob.b).cuda()
    with make_solver(G, prob, "csr", precond) as Sc, make_solver(G, prob, "stencil", precond) as Ss:
        for variant in ("hs", "pr", "m", "cgcg"):
            for k in (1, 2, 3, 4):
                xc = Sc.solve(b, variant=variant, tol=0.0, maxit=k).x.cpu().numpy()
                xs = Ss.solve(b, variant=variant, tol=0.0, maxit=k).x.cpu().numpy()
                assert rel(xs, xc) <= 1e-14, (variant, k, rel(xs, xc))
            band = OracleBand(variant, A, prob.b, d, 20)
            for k in (7, 15, 20):
                if band.determined(k):
                    xs = Ss.solve(b, variant=variant, tol=0.0, maxit=k).x.cpu().numpy()
                    assert band.dist_x(k, xs) <= band.bar_x(k), (variant, k)
