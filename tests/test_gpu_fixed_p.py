"""The block fixed-point copy of p in the constant-stencil product sweeps.

On the graph path (n above the persistent bound, forced here with
PRCG_PERSIST_MAX=0) HS-CG, PR-CG and M-CG on a constant-coefficient stencil
store, in the sweep that forms p, a 64-bit fixed-point copy of p with one
scale per vector, and the product sweep adds the neighbour values with
integer adds.  pipe-PR-CG and pipe-M-CG do the same with copies of r~
and s~ (one pair per buffer; their first two sweeps use the per-row sums).
With an integer diagonal c in [1, 8] (Poisson, or an
integer shift) the product row c P_i - sum P_j is formed entirely in 64-bit
integers; PRCG_NO_INT_DIAG=1 keeps the FP64 FMA c p_i - sum.  Checked here:
the sweeps really read the copy (the library's counter), the iterates match the oracle (Algorithms 1, 2 and 3) under the
parity bar and the per-row fixed-point path (PRCG_NO_FIXED_P=1) to 1e-12,
converged solves stop within one iteration of the oracle, and a right-hand
side scaled by 2^400 or 2^-400 gives exactly the scaled iterates (the scale
S moves by exactly -400 or +400, including negative S).
"""
import numpy as np
import pytest

import oracle as O
import problems as P
from gpu_common import ITER_TOL, OracleBand, case, csr_matrix, rel

pytestmark = pytest.mark.gpu

VARIANTS = ("hs", "pr", "m", "pr_norecompute", "pipe_pr", "pipe_m")
ORACLE = {"hs": ("hs", {}), "pr": ("pr", {}), "m": ("m", {}),
          "pr_norecompute": ("pr", {"recompute_nu": False}),
          "pipe_pr": ("pipe_pr", {}), "pipe_m": ("pipe_m", {})}


def _want_fixed(v, k):
    """Product sweeps of a k-iteration solve that read a fixed-point copy:
    HS-CG forms p_k after its first product; the pipelined sweeps store the
    copies from their second sweep on and read them from their third."""
    if v == "hs":
        return k - 1
    if v.startswith("pipe"):
        return max(0, k - 2)
    return k


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


def _fixed_sweeps(S):
    from paper_1905_01549_gb300 import binding
    return binding.prcg_last_fixed_sweeps(S.handle)


@pytest.mark.parametrize("name", ["poisson3d_ragged", "shifted2d", "poisson2d_64"])
@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_fixed_p_iterates_match_oracle_and_per_row_path(G, name, precond, monkeypatch):
    import torch
    monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = case(name)
    A = csr_matrix(prob)
    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
    b = torch.from_numpy(prob.b).cuda()
    xs = {}
    for env in ("0", "1"):
        monkeypatch.setenv("PRCG_NO_FIXED_P", env)
        with G.Solver.from_stencil(prob.dims, diag_shift=prob.shift, precond=precond) as S:
            for v in VARIANTS:
                for k in (1, 2, 7, 20):
                    res = S.solve(b, variant=v, tol=0.0, maxit=k, history=True)
                    assert res.iters == k
                    want = _want_fixed(v, k) if env == "0" else 0
                    assert _fixed_sweeps(S) == want, (v, k, env, _fixed_sweeps(S))
                    xs[(env, v, k)] = (res.x.cpu().numpy(), res.hist)
    for v in VARIANTS:
        ov, kw = ORACLE[v]
        band = OracleBand(ov, A, prob.b, d, 20, **kw)
        for k in (1, 2, 7, 20):
            xf, hf = xs[("0", v, k)]
            xr, _ = xs[("1", v, k)]
            assert rel(xf, xr) <= 1e-12, (v, k, rel(xf, xr))
            assert band.determined(k) and band.bar_x(k) <= 1e-7
            assert band.dist_x(k, xf) <= band.bar_x(k), (v, k, band.dist_x(k, xf))
            ok, worst = band.hist_ok(k, hf, 1e-9)
            assert ok, (v, k, worst)


@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_fixed_p_converged_solves(G, precond, monkeypatch):
    import torch
    monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = P.grid_problem((40, 36, 30), "fixed_p_conv")
    A = csr_matrix(prob)
    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
    b = torch.from_numpy(prob.b).cuda()
    with G.Solver.from_stencil(prob.dims, precond=precond) as S:
        for v in ("hs", "pr", "m", "pipe_pr"):
            ref = O.solve(v, A, prob.b, d=d, tol=1e-10, maxit=4000)
            res = S.solve(b, variant=v, tol=1e-10, maxit=4000, true_relres=True)
            assert res.status == ref.status == O.OK
            assert abs(res.iters - ref.iters) <= 1, (v, res.iters, ref.iters)
            assert _fixed_sweeps(S) >= res.iters - 2
            assert res.true_relres <= 1e-9
            assert rel(res.x.cpu().numpy(), ref.x) <= 1e-8


@pytest.mark.parametrize("shift", [400, -400])
def test_fixed_p_scale_invariance(G, shift, monkeypatch):
    """b 2^e gives x 2^e bit for bit: every FP64 operation scales exactly and
    the fixed-point scale moves by -e, so the integers P_i are unchanged."""
    import torch
    monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = case("poisson3d_ragged")
    with G.Solver.from_stencil(prob.dims, precond="jacobi") as S:
        for v in ("hs", "pr", "pipe_pr"):
            base = S.solve(torch.from_numpy(prob.b).cuda(), variant=v, tol=0.0, maxit=25)
            n0 = _fixed_sweeps(S)
            scaled = S.solve(torch.from_numpy(np.ldexp(prob.b, shift)).cuda(), variant=v,
                             tol=0.0, maxit=25)
            assert _fixed_sweeps(S) == n0 > 0
            assert np.array_equal(np.ldexp(base.x.cpu().numpy(), shift), scaled.x.cpu().numpy())


def test_fixed_p_edge_cases(G, monkeypatch):
    """b = 0, maxit 0 and 1, an exact x_0 and a NaN in b on the graph path."""
    import torch
    monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    dims = (13, 9, 7)
    x0 = np.random.default_rng(4).integers(-5, 6, 13 * 9 * 7).astype(np.float64)
    b = P.stencil_apply(dims, x0)   # integers: r_0 = 0 exactly
    with G.Solver.from_stencil(dims) as S:
        for v in ("hs", "pr", "m", "pipe_pr"):
            z = torch.ones(x0.size, dtype=torch.float64, device="cuda")
            res = S.solve(torch.zeros_like(z), x0=z, variant=v, tol=1e-10, maxit=50)
            assert res.status == G.PRCG_OK and res.iters == 0 and float(z.abs().max()) == 0.0
            res = S.solve(torch.from_numpy(b).cuda(), x0=torch.from_numpy(x0.copy()).cuda(),
                          variant=v, tol=1e-12, maxit=50)
            assert res.status == G.PRCG_OK and res.iters == 0
            for m in (0, 1):
                res = S.solve(torch.from_numpy(b + 1.0).cuda(), variant=v, tol=1e-12, maxit=m)
                assert res.status == G.PRCG_NOT_CONVERGED and res.iters == m
            bad = b.copy()
            bad[7] = np.nan
            res = S.solve(torch.from_numpy(bad).cuda(), variant=v, tol=1e-10, maxit=50)
            assert res.status == G.PRCG_BREAKDOWN and res.iters == 0


@pytest.mark.parametrize("dims,shift", [((20, 11, 7), 0.0), ((20, 11, 7), 2.0), ((20, 11, 7), 3.0),
                                        ((21, 10, 6), 1.0), ((34, 18), 0.0), ((33, 17), 4.0)])
@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_integer_diagonal_row(G, dims, shift, precond, monkeypatch):
    """c = 2 dim + shift: 6, 8 and 7 (3D) and 4 and 8 (2D, 8 at the limit)
    take the integer row, 9 (3D, shift 3) keeps the FMA; the two forms of
    the row agree to 1e-12 over 20 iterations and both follow the oracle
    (Algorithms 1, 2 and 3) within the parity bar."""
    import torch
    monkeypatch.setenv("PRCG_PERSIST_MAX", "0")
    prob = P.grid_problem(dims, "int_diag", shift=shift)
    A = csr_matrix(prob)
    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
    b = torch.from_numpy(prob.b).cuda()
    xs = {}
    for env in ("0", "1"):
        monkeypatch.setenv("PRCG_NO_INT_DIAG", env)
        with G.Solver.from_stencil(prob.dims, diag_shift=prob.shift, precond=precond) as S:
            c = 2 * len(dims) + shift
            assert S.int_diagonal == (int(c) if env == "0" and c <= 8 else 0)
            for v in ("hs", "pr", "pipe_pr"):
                for k in (1, 5, 20):
                    res = S.solve(b, variant=v, tol=0.0, maxit=k, history=True)
                    assert res.iters == k
                    assert _fixed_sweeps(S) == _want_fixed(v, k)
                    xs[(env, v, k)] = (res.x.cpu().numpy(), res.hist)
    for v in ("hs", "pr", "pipe_pr"):
        band = OracleBand(v, A, prob.b, d, 20)
        for k in (1, 5, 20):
            xi, hi = xs[("0", v, k)]
            xf, _ = xs[("1", v, k)]
            assert rel(xi, xf) <= 1e-12, (v, k, rel(xi, xf))
            assert band.determined(k) and band.dist_x(k, xi) <= band.bar_x(k), (v, k)
            ok, worst = band.hist_ok(k, hi, 1e-9)
            assert ok, (v, k, worst)
