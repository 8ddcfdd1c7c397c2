"""Convergence study of the GPU variants, following Section 4's method.

The paper compares the variants by the A-norm error of their iterates,
||x* - x_k||_A / ||x* - x_0||_A: Table 2 lists, per matrix and variant, the
number of iterations needed to reduce it by a factor 10^5 and the smallest
value it reaches (the maximal attainable accuracy).  This module computes
the same two statistics for the library's GPU variants.

The GPU path is deterministic (fixed-order reductions), so the iterate x_k
of one long run is exactly the result of a solve stopped at maxit = k.  The
study therefore reruns a variant with maxit = 0, 1, ..., K and measures each
returned iterate with the library's own operator (``Solver.error_anorm``,
one GPU sweep).  The cost is O(K^2) iterations, which suits the model
problems of Section 4 (tens to a few hundred iterations); ``stride`` thins
the grid of k for longer runs.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Iterable, Optional

import numpy as np

from . import PRCG_BREAKDOWN, Solver


@dataclasses.dataclass
class ErrorCurve:
    k: np.ndarray             # iteration numbers at which the error was measured
    err: np.ndarray           # ||x* - x_k||_A / ||x* - x_0||_A
    breakdown_at: Optional[int]   # first k at which the variant reported breakdown

    def iterations_to(self, reduction: float = 1e5) -> Optional[int]:
        """First measured k with err <= 1 / reduction (None if never)."""
        hit = np.nonzero(self.err <= 1.0 / reduction)[0]
        return int(self.k[hit[0]]) if len(hit) else None

    def min_log10(self) -> float:
        """log10 of the smallest error reached (Table 2's accuracy column)."""
        m = float(self.err.min())
        return math.log10(m) if m > 0 else -math.inf


def error_curve(S: Solver, b, x_star, variant: str, kmax: int, stride: int = 1,
                x0=None) -> ErrorCurve:
    """A-norm error of the iterates x_0 .. x_kmax of one run of `variant`.

    b, x_star, x0: CUDA tensors (or host arrays) of length S.n; x0 defaults
    to zero.  Stops early once the variant breaks down (later iterates would
    repeat the last one)."""
    import torch
    if x0 is None:
        x0 = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    x0 = x0 if hasattr(x0, "is_cuda") else torch.as_tensor(np.asarray(x0, dtype=np.float64)).cuda()
    e0 = S.error_anorm(x_star, x0)
    if not e0 > 0.0:
        raise ValueError("x0 equals x*: the relative error is undefined")
    ks, errs = [], []
    breakdown_at = None
    for k in range(0, kmax + 1, stride):
        x = x0.clone()
        res = S.solve(b, x0=x, variant=variant, tol=0.0, maxit=k)
        ks.append(res.iters)
        errs.append(S.error_anorm(x_star, x) / e0)
        if res.status == PRCG_BREAKDOWN:
            breakdown_at = res.iters
            break
    return ErrorCurve(np.asarray(ks), np.asarray(errs), breakdown_at)


def study(S: Solver, b, x_star, variants: Iterable[str], kmax: int, stride: int = 1,
          reduction: float = 1e5) -> Dict[str, dict]:
    """Table 2's statistics for each variant: iterations to a `reduction`-fold
    A-norm error reduction and the minimum log10 error."""
    out = {}
    for v in variants:
        c = error_curve(S, b, x_star, v, kmax, stride)
        out[v] = {"iters_to_reduction": c.iterations_to(reduction),
                  "min_log10_err": c.min_log10(),
                  "breakdown_at": c.breakdown_at,
                  "measured_iterations": int(c.k[-1])}
    return out
