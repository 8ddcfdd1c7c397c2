"""GB300-native predict-and-recompute conjugate gradients (Chen & Carson).

The solver is the CUDA library libprcg.so (C ABI in include/prcg.h); this
package loads it with ctypes (``binding``) and wraps a context in a small
``Solver`` class that takes torch tensors.  PyTorch is used only to hold
device memory and name streams.  Importing the package fails if the library
has not been built (``paper_1905_01549_gb300.build.build()``).
"""
from __future__ import annotations

import dataclasses
import os
from typing import Optional, Sequence

import numpy as np

from . import binding
from .binding import (PRCG_BREAKDOWN, PRCG_NOT_CONVERGED, PRCG_OK, PrcgError,  # noqa: F401
                      VARIANT_IDS)

binding.load()

PRECONDS = {"none": binding.PRCG_PRECOND_NONE, "jacobi": binding.PRCG_PRECOND_JACOBI}


@dataclasses.dataclass
class SolveResult:
    x: object                 # x_K (same kind of array as the x passed / a new CUDA tensor)
    iters: int                # K
    status: int               # PRCG_OK / PRCG_NOT_CONVERGED / PRCG_BREAKDOWN
    hist: Optional[np.ndarray]  # ||r_k|| / ||b||, k = 0..K
    true_relres: Optional[float]
    init_ms: float
    loop_ms: float
    trace: Optional[np.ndarray] = None   # (K + 1, 10) scalars per iteration, see prcg.h


def _torch():
    import torch
    return torch


class Solver:
    """One library context (operator + preconditioner) for repeated solves."""

    def __init__(self, handle: int, n: int):
        self.handle = handle
        self.n = n

    @classmethod
    def from_csr(cls, row_ptr, col_idx, vals, precond: str = "none", stream=None) -> "Solver":
        n = len(row_ptr) - 1
        nnz = len(vals)
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32) if isinstance(row_ptr, np.ndarray) else row_ptr
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32) if isinstance(col_idx, np.ndarray) else col_idx
        vals = np.ascontiguousarray(vals, dtype=np.float64) if isinstance(vals, np.ndarray) else vals
        h = binding.prcg_create_csr(n, nnz, row_ptr, col_idx, vals, PRECONDS[precond], stream)
        return cls(h, n)

    @classmethod
    def from_stencil(cls, dims: Sequence[int], face_coeff=None, diag_shift: float = 0.0,
                     precond: str = "none", stream=None) -> "Solver":
        dims = tuple(int(d) for d in dims)
        nx, ny = dims[0], dims[1]
        nz = dims[2] if len(dims) == 3 else 1
        if isinstance(face_coeff, np.ndarray):
            face_coeff = np.ascontiguousarray(face_coeff, dtype=np.float64)
        h = binding.prcg_create_stencil(len(dims), nx, ny, nz, face_coeff, diag_shift,
                                        PRECONDS[precond], stream)
        return cls(h, nx * ny * nz)

    @classmethod
    def from_dense(cls, A, precond: str = "none", stream=None) -> "Solver":
        """Dense symmetric positive definite A (n x n numpy array or CUDA
        tensor, row-major); the context keeps its own copy."""
        n = int(A.shape[0])
        if A.shape != (n, n):
            raise ValueError("A must be square")
        if isinstance(A, np.ndarray):
            A = np.ascontiguousarray(A, dtype=np.float64)
        h = binding.prcg_create_dense(n, A, PRECONDS[precond], stream)
        return cls(h, n)

    @property
    def jacobi_form(self) -> str:
        """How the preconditioner is applied: "none", "scalar" or "vector"."""
        return ("none", "scalar", "vector")[binding.prcg_jacobi_form(self.handle)]

    @property
    def int_diagonal(self) -> int:
        """A constant stencil's integer diagonal (1..8) if its fixed-point product
        rows run in integers, else 0."""
        return binding.prcg_int_diagonal(self.handle)

    def solve(self, b, x0=None, variant: str = "pr", tol: float = 1e-10,
              maxit: Optional[int] = None, history: bool = False,
              true_relres: bool = False, trace: bool = False) -> SolveResult:
        """Solve A x = b.  b / x0 may be CUDA tensors, CPU tensors or numpy arrays.

        Without x0 a zero CUDA tensor is used and returned as x; with x0 the
        result overwrites x0 in place."""
        torch = _torch()
        if maxit is None:
            maxit = 2 * self.n
        if isinstance(b, np.ndarray):
            b = np.ascontiguousarray(b, dtype=np.float64)
        x = x0 if x0 is not None else torch.zeros(self.n, dtype=torch.float64, device="cuda")
        hist = np.empty(maxit + 1) if history else None
        if trace:
            binding.prcg_trace_enable(self.handle, True)
        try:
            status, iters, trr = binding.prcg_solve(self.handle, VARIANT_IDS[variant], b, x, tol,
                                                    maxit, hist, true_relres)
            tr = binding.prcg_trace_get(self.handle, maxit + 2) if trace else None
        finally:
            if trace:
                binding.prcg_trace_enable(self.handle, False)
        init_ms, loop_ms, _ = binding.prcg_last_timing(self.handle)
        return SolveResult(x, iters, status, None if hist is None else hist[:iters + 1], trr,
                           init_ms, loop_ms, tr)

    def solve_refined_fp32(self, b, x0=None, tol: float = 1e-8, max_outer: int = 30,
                           inner_tol: float = 1e-4, inner_maxit: Optional[int] = None):
        """FP32 PR-CG inner solves + FP64 iterative refinement.  Returns
        (x, status, outer steps, inner iterations, true relres, outer history, ms)."""
        torch = _torch()
        x = x0 if x0 is not None else torch.zeros(self.n, dtype=torch.float64, device="cuda")
        if inner_maxit is None:
            inner_maxit = 2 * self.n
        hist = np.zeros(max_outer + 1)
        status, outer, inner, trr = binding.prcg_solve_f32_refined(
            self.handle, b, x, tol, max_outer, inner_tol, inner_maxit, hist)
        _, loop_ms, _ = binding.prcg_last_timing(self.handle)
        return x, status, outer, inner, trr, hist[:outer + 1], loop_ms

    def error_anorm(self, x_star, x) -> float:
        """||x* - x||_A with this context's operator (Section 4's error measure)."""
        if isinstance(x_star, np.ndarray):
            x_star = np.ascontiguousarray(x_star, dtype=np.float64)
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
        return binding.prcg_error_anorm(self.handle, x_star, x)

    def check_guards(self) -> int:
        """Corrupted guard words (prcg_check_guards); 0 when every kernel
        stayed within its buffers."""
        return binding.prcg_check_guards(self.handle)

    def close(self):
        if self.handle:
            h, self.handle = self.handle, None
            try:
                # test runs set PRCG_CHECK_GUARDS=1: every context is checked
                # for out-of-bounds writes before it is freed
                if os.environ.get("PRCG_CHECK_GUARDS") == "1":
                    bad = binding.prcg_check_guards(h)
                    if bad:
                        raise PrcgError(binding.PRCG_ERR_CUDA,
                                        f"{bad} guard words corrupted (out-of-bounds write)")
            finally:
                binding.prcg_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchedSolver:
    """Many shifted 2D 5-point systems of uneven size solved by one persistent
    PR-CG launch (C ABI prcg_batched_*)."""

    def __init__(self, nx, ny, shift, precond: str = "none", stream=None):
        self.nx = np.asarray(nx, dtype=np.int32)
        self.ny = np.asarray(ny, dtype=np.int32)
        self.shift = np.asarray(shift, dtype=np.float64)
        self.precond = PRECONDS[precond]
        self.sizes = self.nx.astype(np.int64) * self.ny
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)])
        self.total = int(self.offsets[-1])
        self.handle = binding.prcg_batched_create(self.nx, self.ny, self.shift, self.precond, stream)

    def configure(self, cluster: int, threads: int):
        binding.prcg_batched_configure(self.handle, cluster, threads)

    def configure_split(self, nbig: int, big, rest):
        """The nbig costliest systems on clusters big = (cluster, threads),
        the others on a concurrent launch of rest = (cluster, threads)."""
        binding.prcg_batched_configure_split(self.handle, nbig, big[0], big[1], rest[0], rest[1])

    def config(self):
        return binding.prcg_batched_config(self.handle)

    def split(self):
        """(nbig, cluster, threads, clusters) of the second launch; zeros if not split."""
        return binding.prcg_batched_split(self.handle)

    def tune(self, b, x0=None, tol: float = 1e-8, maxit: int = 100000, **kw):
        from . import autotune
        torch = _torch()
        if x0 is None:
            x0 = torch.zeros(self.total, dtype=torch.float64, device="cuda")
        key = autotune.batch_key(self.nx, self.ny, self.shift, self.precond, tol,
                                 torch.cuda.get_device_name())
        return autotune.tune(self.handle, b, x0, tol, maxit, key=key, **kw)

    def solve(self, b, x0=None, tol: float = 1e-8, maxit: int = 100000, true_relres: bool = False):
        """Returns (x, iters[nsys], status[nsys], true_relres[nsys] or None, worst status, ms)."""
        torch = _torch()
        x = x0 if x0 is not None else torch.zeros(self.total, dtype=torch.float64, device="cuda")
        iters = np.zeros(len(self.nx), dtype=np.int32)
        status = np.zeros(len(self.nx), dtype=np.int32)
        trr = np.zeros(len(self.nx)) if true_relres else None
        worst = binding.prcg_batched_solve(self.handle, b, x, tol, maxit, iters, status, trr)
        return x, iters, status, trr, worst, binding.prcg_batched_last_ms(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            binding.prcg_batched_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
