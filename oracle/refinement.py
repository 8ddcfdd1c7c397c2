"""Oracle of the mixed-precision form: FP32 PR-CG inner solves inside FP64
iterative refinement.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's experiments are all FP64; this form is an extension.  The inner
solve is the oracle's own PR-CG (Algorithm 2) run on float32 arrays: numpy
keeps the vectors, the matrix and the inner products in float32 while the
scalars alpha, beta, nu' stay Python floats (FP64), which is the precision
split the GPU form uses.  The outer loop is classical iterative refinement:
t = b - A x in FP64, stop when ||t|| / ||b|| <= tol, solve A d = t / ||t||
in FP32 to inner_tol, x += ||t|| d in FP64; stop also when a step does not
reduce the true residual.
"""
from __future__ import annotations

import numpy as np

from .cg_variants import NOT_CONVERGED, OK, BREAKDOWN, as_operator, pr_cg


def refined_fp32(A, b, tol=1e-8, max_outer=30, inner_tol=1e-4, inner_maxit=None, d=None):
    """Returns (x, status, outer steps, inner iterations, history of ||t||/||b||)."""
    n = b.shape[0]
    if inner_maxit is None:
        inner_maxit = 2 * n
    A64 = as_operator(A)
    if isinstance(A, np.ndarray):
        A32 = A.astype(np.float32)
    else:
        A32 = A.astype(np.float32)
    d32 = None if d is None else np.asarray(d, dtype=np.float32)
    x = np.zeros(n)
    bn = float(np.linalg.norm(b))
    hist = []
    inner_total = 0
    prev = np.inf
    outer = 0
    while True:
        t = b - A64(x)
        tn = float(np.linalg.norm(t))
        if bn == 0.0:
            hist.append(0.0)
            return np.zeros(n), OK, outer, inner_total, hist
        rel = tn / bn
        hist.append(rel)
        if rel <= tol:
            return x, OK, outer, inner_total, hist
        if outer >= max_outer or not rel < prev:
            return x, NOT_CONVERGED, outer, inner_total, hist
        prev = rel
        rhs = (t / tn).astype(np.float32)
        res = pr_cg(A32, rhs, d=d32, tol=inner_tol, maxit=inner_maxit)
        inner_total += res.iters
        if res.iters == 0:
            return x, BREAKDOWN, outer, inner_total, hist
        x = x + tn * res.x.astype(np.float64)
        outer += 1
