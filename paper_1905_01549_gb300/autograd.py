"""Differentiable solves: torch.autograd.Functions whose backward runs the
adjoint solve on the GPU library.

For x = A^{-1} b with A symmetric positive definite and an upstream gradient
g = dL/dx, the backward pass solves A lambda = g with the same variant and
tolerance (one more prcg_solve on the same context), returns dL/db = lambda
and forms the gradient of A's parameters with a CUDA kernel:
* face coefficients of the diffusion stencil: -(lambda_a - lambda_b)(x_a - x_b)
  per interior face, -lambda_a x_a per boundary face (prcg_grad_faces);
* CSR values: -lambda_i x_j per stored entry (prcg_grad_csr_values).
The forward and adjoint solves run to `tol`; the gradients are as accurate
as those two solves.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import Solver, binding


class _DiffusionSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, faces, b, solver, shift, variant, tol, maxit):
        binding.prcg_update_faces(solver.handle, faces.detach().contiguous(), shift)
        x = torch.zeros_like(b)
        res = solver.solve(b.detach().contiguous(), x0=x, variant=variant, tol=tol, maxit=maxit)
        if res.status != binding.PRCG_OK:
            raise binding.PrcgError(res.status, "forward solve did not converge")
        ctx.solver, ctx.shift, ctx.variant, ctx.tol, ctx.maxit = solver, shift, variant, tol, maxit
        ctx.save_for_backward(faces, x)
        return x

    @staticmethod
    def backward(ctx, g):
        faces, x = ctx.saved_tensors
        S = ctx.solver
        binding.prcg_update_faces(S.handle, faces.detach().contiguous(), ctx.shift)
        lam = torch.zeros_like(x)
        res = S.solve(g.detach().contiguous(), x0=lam, variant=ctx.variant, tol=ctx.tol,
                      maxit=ctx.maxit)
        if res.status != binding.PRCG_OK:
            raise binding.PrcgError(res.status, "adjoint solve did not converge")
        grad_faces = None
        if ctx.needs_input_grad[0]:
            grad_faces = torch.empty_like(faces)
            binding.prcg_grad_faces(S.handle, lam, x, grad_faces)
        grad_b = lam if ctx.needs_input_grad[1] else None
        return grad_faces, grad_b, None, None, None, None, None


class DiffusionSolver:
    """x = A(c)^{-1} b for the variable-coefficient stencil, differentiable in
    the face coefficients c and in b.  One library context per grid."""

    def __init__(self, dims: Sequence[int], precond: str = "jacobi", shift: float = 0.0):
        self.dims = tuple(int(d) for d in dims)
        self.shift = float(shift)
        nf = _face_count(self.dims)
        ones = torch.ones(nf, dtype=torch.float64, device="cuda")
        self.solver = Solver.from_stencil(self.dims, face_coeff=ones, diag_shift=shift,
                                          precond=precond)

    def __call__(self, faces: torch.Tensor, b: torch.Tensor, variant: str = "pr",
                 tol: float = 1e-12, maxit: Optional[int] = None) -> torch.Tensor:
        if maxit is None:
            maxit = 50 * self.solver.n
        return _DiffusionSolve.apply(faces, b, self.solver, self.shift, variant, tol, maxit)

    def close(self):
        self.solver.close()


def _face_count(dims):
    if len(dims) == 2:
        nx, ny = dims
        return ny * (nx + 1) + (ny + 1) * nx
    nx, ny, nz = dims
    return nz * ny * (nx + 1) + nz * (ny + 1) * nx + (nz + 1) * ny * nx


def csr_solve(vals: torch.Tensor, b: torch.Tensor, row_ptr, col_idx, precond: str = "jacobi",
              variant: str = "pr", tol: float = 1e-12, maxit: Optional[int] = None):
    """x = A^{-1} b for A given by CSR (row_ptr, col_idx, vals), differentiable
    in vals (stored entries) and b."""
    if maxit is None:
        maxit = 50 * (len(row_ptr) - 1)
    return _CSRSolveV.apply(vals, b, row_ptr, col_idx, precond, variant, tol, maxit)


class _CSRSolveV(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, row_ptr, col_idx, precond, variant, tol, maxit):
        S = Solver.from_csr(row_ptr, col_idx, vals.detach().contiguous(), precond=precond)
        x = torch.zeros_like(b)
        res = S.solve(b.detach().contiguous(), x0=x, variant=variant, tol=tol, maxit=maxit)
        if res.status != binding.PRCG_OK:
            S.close()
            raise binding.PrcgError(res.status, "forward solve did not converge")
        ctx.solver, ctx.variant, ctx.tol, ctx.maxit = S, variant, tol, maxit
        ctx.nnz = int(vals.numel())
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        S = ctx.solver
        lam = torch.zeros_like(x)
        res = S.solve(g.detach().contiguous(), x0=lam, variant=ctx.variant, tol=ctx.tol,
                      maxit=ctx.maxit)
        if res.status != binding.PRCG_OK:
            raise binding.PrcgError(res.status, "adjoint solve did not converge")
        grad_vals = None
        if ctx.needs_input_grad[0]:
            grad_vals = torch.empty(ctx.nnz, dtype=torch.float64, device=x.device)
            binding.prcg_grad_csr_values(S.handle, lam, x, grad_vals)
        S.close()
        return grad_vals, (lam if ctx.needs_input_grad[1] else None), None, None, None, None, None, None
