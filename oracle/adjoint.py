"""Oracle of the adjoint gradients of x = A^{-1} b.  TEST INFRASTRUCTURE ONLY.

The paper has no gradients; this is the differentiable form's reference.
For a loss L(x) with g = dL/dx and A symmetric positive definite:
lambda = A^{-1} g, dL/db = lambda, and dL/dA = -lambda x^T restricted to the
stored entries.  For the face-coefficient operator A = sum_f c_f
(e_a - e_b)(e_a - e_b)^T (e_b = 0 on boundary faces):
dL/dc_f = -(lambda_a - lambda_b)(x_a - x_b), or -lambda_a x_a on the boundary.
Both solves use the oracle's PR-CG (Algorithm 2)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .cg_variants import jacobi_inverse_diagonal, pr_cg


def _csr(rp, ci, v, n):
    return sp.csr_matrix((v, ci, rp), shape=(n, n))


def solve_pair(A, b, g_of_x, tol=1e-13, precond=True):
    d = jacobi_inverse_diagonal(A) if precond else None
    maxit = 50 * A.shape[0]
    x = pr_cg(A, b, d=d, tol=tol, maxit=maxit).x
    g = g_of_x(x)
    lam = pr_cg(A, g, d=d, tol=tol, maxit=maxit).x
    return x, lam


def face_gradient(dims, lam, x):
    """dL/dc_f in the concatenated face layout (x-, y-, (z-) faces)."""
    if len(dims) == 2:
        nx, ny = dims
        nz = 1
    else:
        nx, ny, nz = dims
    X = x.reshape(nz, ny, nx)
    Lm = lam.reshape(nz, ny, nx)
    out = []
    # x-faces (nz, ny, nx+1)
    gx = np.zeros((nz, ny, nx + 1))
    gx[:, :, 1:nx] = -(Lm[:, :, :-1] - Lm[:, :, 1:]) * (X[:, :, :-1] - X[:, :, 1:])
    gx[:, :, 0] = -Lm[:, :, 0] * X[:, :, 0]
    gx[:, :, nx] = -Lm[:, :, nx - 1] * X[:, :, nx - 1]
    out.append(gx)
    gy = np.zeros((nz, ny + 1, nx))
    gy[:, 1:ny, :] = -(Lm[:, :-1, :] - Lm[:, 1:, :]) * (X[:, :-1, :] - X[:, 1:, :])
    gy[:, 0, :] = -Lm[:, 0, :] * X[:, 0, :]
    gy[:, ny, :] = -Lm[:, ny - 1, :] * X[:, ny - 1, :]
    out.append(gy)
    if len(dims) == 3:
        gz = np.zeros((nz + 1, ny, nx))
        gz[1:nz] = -(Lm[:-1] - Lm[1:]) * (X[:-1] - X[1:])
        gz[0] = -Lm[0] * X[0]
        gz[nz] = -Lm[nz - 1] * X[nz - 1]
        out.append(gz)
    return np.concatenate([o.ravel() for o in out])


def csr_value_gradient(rp, ci, lam, x):
    """dL/da_e = -lambda_i x_{col(e)} for every stored entry e of row i."""
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return -lam[rows] * x[ci]
