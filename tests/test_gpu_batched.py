"""Batched persistent PR-CG vs the oracle, system by system.

Every system of a small uneven batch (shifted 2D 5-point operators) is
compared with its own single-system oracle PR-CG solve at the same
tolerance; several cluster / CTA configurations must agree with it."""
import numpy as np
import pytest

import oracle as O
import problems as P
from gpu_common import rel

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


def _batch(count=24, lo=8, hi=80):
    spec = P.batch_spec(count, lo, hi, tag="t_batch")
    systems = [spec.system(i) for i in range(count)]
    # a few rectangular grids and the degenerate 1 x 1 case
    systems[3] = P.grid_problem((17, 5), "t_rect", shift=0.02, with_csr=False, rhs="uniform")
    if count > 7:
        systems[7] = P.grid_problem((1, 1), "t_one", shift=0.0, with_csr=False, rhs="uniform")
    return systems


def _oracle(sysp, precond):
    import scipy.sparse as sp
    rp, ci, v = P.stencil_csr(sysp.dims, None, sysp.shift)
    A = sp.csr_matrix((v, ci, rp), shape=(sysp.n, sysp.n))
    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
    return A, O.pr_cg(A, sysp.b, d=d, tol=TOL, maxit=20000)


@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_batched_matches_single_system_oracle(G, precond):
    import torch
    systems = _batch()
    nx = [s.dims[0] for s in systems]
    ny = [s.dims[1] for s in systems]
    shift = [s.shift for s in systems]
    B = G.BatchedSolver(nx, ny, shift, precond=precond)
    b = torch.from_numpy(np.concatenate([s.b for s in systems])).cuda()
    refs = [_oracle(s, precond) for s in systems]
    results = {}
    for cluster, threads in [(1, 256), (1, 1024), (2, 128), (4, 256), (8, 64)]:
        B.configure(cluster, threads)
        x, iters, status, trr, worst, ms = B.solve(b, tol=TOL, true_relres=True)
        assert worst == G.PRCG_OK and np.all(status == 0), (cluster, threads)
        xs = x.cpu().numpy()
        for i, (s, (A, ref)) in enumerate(zip(systems, refs)):
            xi = xs[B.offsets[i]:B.offsets[i + 1]]
            assert abs(int(iters[i]) - ref.iters) <= max(1, 0.05 * ref.iters), (i, iters[i], ref.iters)
            assert rel(xi, ref.x) <= 1e-6, (i, rel(xi, ref.x))
            assert trr[i] <= 2 * TOL and O.true_relres(A, s.b, xi) <= 2 * TOL
        results[(cluster, threads)] = xs
        # the same configuration again: bitwise identical
        x2, *_ = B.solve(b, tol=TOL)
        assert np.array_equal(x2.cpu().numpy(), xs)
    B.close()


@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_split_launch_matches_single_system_oracle(G, precond):
    """The costliest systems on one launch, the rest on a concurrent second
    launch: every system still matches its own oracle solve."""
    import torch
    systems = _batch()
    B = G.BatchedSolver([s.dims[0] for s in systems], [s.dims[1] for s in systems],
                        [s.shift for s in systems], precond=precond)
    b = torch.from_numpy(np.concatenate([s.b for s in systems])).cuda()
    refs = [_oracle(s, precond) for s in systems]
    for nbig, big, rest in [(3, (16, 256), (4, 128)), (6, (8, 512), (1, 256)),
                            (23, (2, 64), (1, 64))]:
        B.configure_split(nbig, big, rest)
        assert B.split()[:3] == (nbig,) + rest and B.config()[:2] == big
        x, iters, status, trr, worst, ms = B.solve(b, tol=TOL, true_relres=True)
        assert worst == G.PRCG_OK and np.all(status == 0), (nbig, big, rest)
        xs = x.cpu().numpy()
        for i, (s, (A, ref)) in enumerate(zip(systems, refs)):
            xi = xs[B.offsets[i]:B.offsets[i + 1]]
            assert abs(int(iters[i]) - ref.iters) <= max(1, 0.05 * ref.iters), (i, iters[i])
            assert rel(xi, ref.x) <= 1e-6 and trr[i] <= 2 * TOL, i
        x2, *_ = B.solve(b, tol=TOL)
        assert np.array_equal(x2.cpu().numpy(), xs)
    B.configure(1, 256)
    assert B.split() == (0, 0, 0, 0)
    from paper_1905_01549_gb300 import binding
    for nbig in (0, len(systems)):
        with pytest.raises(binding.PrcgError):
            B.configure_split(nbig, (8, 256), (1, 256))
    assert B.config()[:2] == (1, 256) and B.split()[0] == 0   # a refused split changes nothing
    B.close()


def test_batched_zero_rhs_maxit_and_host_buffers(G):
    import torch
    systems = _batch(6)
    nx = [s.dims[0] for s in systems]
    ny = [s.dims[1] for s in systems]
    B = G.BatchedSolver(nx, ny, [s.shift for s in systems])
    bh = np.concatenate([s.b for s in systems])
    bh[B.offsets[2]:B.offsets[3]] = 0.0          # one zero right-hand side
    xh = np.ones(B.total)                          # x_0 = 1 (host buffers)
    iters = np.zeros(6, dtype=np.int32)
    status = np.zeros(6, dtype=np.int32)
    from paper_1905_01549_gb300 import binding
    worst = binding.prcg_batched_solve(B.handle, bh, xh, TOL, 20000, iters, status)
    assert worst == G.PRCG_OK
    assert iters[2] == 0 and np.all(xh[B.offsets[2]:B.offsets[3]] == 0.0)
    worst = binding.prcg_batched_solve(B.handle, bh, np.zeros(B.total), TOL, 3, iters, status)
    assert worst == G.PRCG_NOT_CONVERGED
    assert np.all(iters[[0, 1, 3, 4, 5]] <= 3)
    B.close()


def test_autotuner_picks_and_caches(G, tmp_path):
    import torch
    from paper_1905_01549_gb300 import autotune
    systems = _batch(16)
    B = G.BatchedSolver([s.dims[0] for s in systems], [s.dims[1] for s in systems],
                        [s.shift for s in systems])
    b = torch.from_numpy(np.concatenate([s.b for s in systems])).cuda()
    cache = str(tmp_path / "tune.json")
    c, t, ms, table = B.tune(b, cache_path=cache, candidates=((1, 256), (2, 256), (4, 128)),
                             splits=())
    assert (c, t) in [(1, 256), (2, 256), (4, 128)] and ms > 0
    assert B.config()[:2] == (c, t)
    B.configure(1, 64)
    c2, t2, _, _ = B.tune(b, cache_path=cache)        # from the cache, no re-timing
    assert (c2, t2) == (c, t) and B.config()[:2] == (c, t)
    B.close()
