"""Adjoint-solve autograd: GPU gradients vs the oracle's adjoint gradients
(1e-9 relative, both from solves at 1e-13) and vs central finite differences
of GPU solves (h = 1e-6).  The finite differences divide loss differences of
~1e-8 by 2h: a solve error of ~1e-12 in the loss moves them by ~1e-6
absolute, so they are held to 1e-4 relative of max(|fd|, 1e-2 max|grad|)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1905_01549_gb300 as G
    return G


@pytest.mark.parametrize("dims", [(24, 19), (9, 7, 6)])
def test_face_and_rhs_gradients(G, dims):
    import torch
    from paper_1905_01549_gb300.autograd import DiffusionSolver
    rng = np.random.default_rng(12)
    faces = P.face_coefficients(dims, 2.0, rng)
    ff = P.flat_faces(faces)
    n = int(np.prod(dims))
    b = rng.uniform(-1, 1, n)
    xt = rng.standard_normal(n)
    D = DiffusionSolver(dims, precond="jacobi")
    fc = torch.tensor(ff, device="cuda", requires_grad=True)
    bc = torch.tensor(b, device="cuda", requires_grad=True)
    xtc = torch.tensor(xt, device="cuda")
    x = D(fc, bc, tol=1e-13)
    loss = ((x - xtc) ** 2).sum()
    loss.backward()
    gf = fc.grad.cpu().numpy()
    gb = bc.grad.cpu().numpy()
    # oracle adjoint gradient
    rp, ci, v = P.stencil_csr(dims, faces, 0.0)
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    xo, lam = O.adjoint.solve_pair(A, b, lambda x_: 2 * (x_ - xt), tol=1e-13)
    go = O.adjoint.face_gradient(dims, lam, xo)
    assert np.linalg.norm(gf - go) <= 1e-9 * np.linalg.norm(go)
    assert np.linalg.norm(gb - lam) <= 1e-9 * np.linalg.norm(lam)
    # central finite differences through the GPU solver
    def loss_at(fv, bv):
        with torch.no_grad():
            xx = D(torch.tensor(fv, device="cuda"), torch.tensor(bv, device="cuda"), tol=1e-13)
            return float(((xx - xtc) ** 2).sum())
    h = 1e-6
    for f in rng.choice(len(ff), 32, replace=False):
        e = np.zeros_like(ff)
        e[f] = h * max(ff[f], 1.0)    # small coefficients get an absolute step
        fd = (loss_at(ff + e, b) - loss_at(ff - e, b)) / (2 * e[f])
        assert abs(fd - gf[f]) <= 1e-4 * max(abs(fd), 1e-2 * np.abs(gf).max()), (f, fd, gf[f])
    dirn = rng.standard_normal(len(ff)) * ff
    fd = (loss_at(ff + h * dirn, b) - loss_at(ff - h * dirn, b)) / (2 * h)
    assert abs(fd - gf @ dirn) <= 1e-4 * abs(fd)
    db = rng.standard_normal(n)
    fd = (loss_at(ff, b + h * db) - loss_at(ff, b - h * db)) / (2 * h)
    assert abs(fd - gb @ db) <= 1e-4 * abs(fd)
    D.close()


def test_csr_value_gradients(G):
    import torch
    from paper_1905_01549_gb300.autograd import csr_solve
    rng = np.random.default_rng(13)
    dims = (17, 13)
    rp, ci, v = P.stencil_csr(dims, P.face_coefficients(dims, 1.0, rng), 0.0)
    n = len(rp) - 1
    b = rng.uniform(-1, 1, n)
    xt = rng.standard_normal(n)
    vc = torch.tensor(v, device="cuda", requires_grad=True)
    bc = torch.tensor(b, device="cuda", requires_grad=True)
    x = csr_solve(vc, bc, rp, ci, tol=1e-13)
    ((x - torch.tensor(xt, device="cuda")) ** 2).sum().backward()
    A = sp.csr_matrix((v, ci, rp), shape=(n, n))
    xo, lam = O.adjoint.solve_pair(A, b, lambda x_: 2 * (x_ - xt), tol=1e-13)
    go = O.adjoint.csr_value_gradient(rp, ci, lam, xo)
    assert np.linalg.norm(vc.grad.cpu().numpy() - go) <= 1e-9 * np.linalg.norm(go)
    assert np.linalg.norm(bc.grad.cpu().numpy() - lam) <= 1e-9 * np.linalg.norm(lam)


def test_512_diffusion_gradients_vs_oracle(G):
    """The differentiation workload at full size (512^2, sigma = 2)."""
    import torch
    from paper_1905_01549_gb300.autograd import DiffusionSolver
    prob = P.varcoef2d(512, rhs="uniform")
    rng = P.rng_for("grad512_xt")
    xt = rng.standard_normal(prob.n)
    ff = prob.face_array()
    D = DiffusionSolver(prob.dims, precond="jacobi")
    fc = torch.tensor(ff, device="cuda", requires_grad=True)
    bc = torch.tensor(prob.b, device="cuda", requires_grad=True)
    x = D(fc, bc, tol=1e-12)
    ((x - torch.tensor(xt, device="cuda")) ** 2).sum().backward()
    rp, ci, v = prob.csr
    A = sp.csr_matrix((v, ci, rp), shape=(prob.n, prob.n))
    xo, lam = O.adjoint.solve_pair(A, prob.b, lambda x_: 2 * (x_ - xt), tol=1e-12)
    go = O.adjoint.face_gradient(prob.dims, lam, xo)
    assert np.linalg.norm(fc.grad.cpu().numpy() - go) <= 1e-7 * np.linalg.norm(go)
    assert np.linalg.norm(bc.grad.cpu().numpy() - lam) <= 1e-7 * np.linalg.norm(lam)
    D.close()
