"""Shared helpers of the GPU tests: problem cases and oracle-side matrices."""
import math

import numpy as np
import scipy.sparse as sp

import oracle as O
import problems as P


def csr_matrix(prob):
    rp, ci, v = prob.csr
    return sp.csr_matrix((v, ci, rp), shape=(prob.n, prob.n))


def case(name):
    """Small cases that span several 256-row tiles and end in a ragged tile."""
    if name == "poisson2d_64":
        return P.poisson2d_64()
    if name == "poisson3d_ragged":
        return P.grid_problem((21, 13, 11), "t_p3r")
    if name == "varcoef3d_ragged":
        return P.grid_problem((19, 11, 7), "t_vc3r", sigma=2.0)
    if name == "varcoef2d_ragged":
        return P.grid_problem((45, 31), "t_vc2r", sigma=2.0)
    if name == "shifted2d":
        return P.grid_problem((33, 47), "t_sh2", shift=0.05, rhs="uniform")
    if name == "varcoef3d_even":
        # even nx: the products take two rows of a grid line per thread
        return P.grid_problem((20, 11, 7), "t_vc3e", sigma=2.0)
    if name == "poisson3d_nx24":
        # nx a multiple of 4: the FP32 stencil product takes four rows at a time
        return P.grid_problem((24, 13, 11), "t_p3x")
    raise KeyError(name)


CASES = ["poisson2d_64", "poisson3d_ragged", "varcoef3d_ragged", "varcoef2d_ragged", "shifted2d",
         "varcoef3d_even"]
GPU_VARIANTS = ["hs", "pr", "pipe_pr", "m", "pipe_m", "cgcg", "gv"]


def make_solver(G, prob, op, precond):
    if op == "csr":
        rp, ci, v = prob.csr
        return G.Solver.from_csr(rp, ci, v, precond=precond)
    return G.Solver.from_stencil(prob.dims, face_coeff=prob.face_array(), diag_shift=prob.shift,
                                 precond=precond)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _fsum_dot(a, b):
    return math.fsum(a * b)


# Parity bar.  Where the iterates of a variant are well determined by FP64
# arithmetic, the GPU must match the oracle to ITER_TOL.  On ill-conditioned
# systems (unpreconditioned log-normal diffusion, clustered Eq. 4.1 spectra)
# a change of rounding alone moves x_k by far more than 1e-10 after a few
# iterations; there the bar is SPREAD_FACTOR times the oracle's own spread
# over three other roundings of the same algorithm, measured as the GPU's
# distance to the nearest of the four runs, and only as long as that bar
# stays within DETERMINED.  Past that point the iterate is not determined by
# the algorithm to better than 1e-6, and the tests check properties instead
# of elements.
ITER_TOL = 1e-10
SPREAD_FACTOR = 8.0
DETERMINED = 1e-6


def _extended(A, b, d):
    """A, b, d in the platform's extended precision (numpy longdouble)."""
    L = np.longdouble
    if sp.issparse(A):
        A = sp.csr_matrix(A)
        AL = sp.csr_matrix((A.data.astype(L), A.indices, A.indptr), shape=A.shape)
    else:
        AL = np.asarray(A).astype(L)
    return AL, np.asarray(b).astype(L), None if d is None else np.asarray(d).astype(L)


def _reversed_rows(A):
    """The same CSR matrix with every row's entries stored in reverse order:
    scipy's product then sums each row in the opposite order."""
    rp, ci, v = A.indptr, A.indices, A.data
    n = A.shape[0]
    row_of = np.repeat(np.arange(n), np.diff(rp))
    rev = rp[row_of] + rp[row_of + 1] - 1 - np.arange(len(v))
    return sp.csr_matrix((v[rev], ci[rev], rp.copy()), shape=A.shape)


def _alt_operator(A):
    """A product with another rounding order than the oracle's default one."""
    if sp.issparse(A):
        Ar = _reversed_rows(sp.csr_matrix(A))
        return lambda v: Ar @ v
    Af = np.ascontiguousarray(np.asarray(A)[:, ::-1])
    return lambda v: Af @ v[::-1]


class OracleBand:
    """The oracle's run of one variant, plus the same algorithm under three
    other roundings -- exactly rounded inner products; that and every
    product summed in the opposite order; everything in the platform's
    extended precision (longdouble) -- each recording x_k for k <= kmax.

    ``bar_x(k)`` is the elementwise bar at iteration k, ``determined(k)``
    whether it stays within DETERMINED, ``dist_x(k, x)`` the relative
    distance of x from the nearest of the three runs' x_k.
    """

    def __init__(self, variant, A, b, d, kmax, **kw):
        import oracle.cg_variants as CV
        self.kmax = kmax
        self.ref = O.solve(variant, A, b, d=d, tol=0.0, maxit=kmax, record=kmax, **kw)
        saved = CV._dot
        CV._dot = lambda u, v: saved(u, v) if u.dtype == object else _fsum_dot(u, v)
        try:
            alt1 = O.solve(variant, A, b, d=d, tol=0.0, maxit=kmax, record=kmax, **kw)
            alt2 = O.solve(variant, _alt_operator(A), b, d=d, tol=0.0, maxit=kmax, record=kmax,
                           **kw)
        finally:
            CV._dot = saved
        L = np.longdouble
        CV._dot = lambda u, v: saved(u, v) if u.dtype != L else L(np.dot(u, v))
        try:
            AL, bL, dL = _extended(A, b, d)
            alt3 = O.solve(variant, AL, bL, d=dL, tol=0.0, maxit=kmax, record=kmax, **kw)
        finally:
            CV._dot = saved
        for k, (xk, rk) in enumerate(alt3.iterates):
            alt3.iterates[k] = (np.asarray(xk, dtype=np.float64), np.asarray(rk, dtype=np.float64))
        alt3.hist = [float(h) for h in alt3.hist]
        alt3.scalars = [{f: float(v) for f, v in sc.items()} for sc in alt3.scalars]
        self.alts = [alt1, alt2, alt3]
        self.runs = [self.ref] + self.alts

    def x(self, k):
        return self.ref.iterates[k][0]

    def spread_x(self, k):
        return max(rel(a.iterates[k][0], self.x(k)) for a in self.alts)

    def bar_x(self, k):
        return max(ITER_TOL, SPREAD_FACTOR * self.spread_x(k))

    def determined(self, k):
        return self.bar_x(k) <= DETERMINED

    def dist_x(self, k, x):
        return min(rel(x, r.iterates[k][0]) for r in self.runs)

    def hist_bars(self, k, floor):
        """Per-entry relative bars of ||r_j|| / ||b||, j = 0..k (NaN where the
        entry, or x_j, is not determined to DETERMINED)."""
        h = np.asarray(self.ref.hist[:k + 1])
        spread = np.zeros(k + 1)
        for a in self.alts:
            ha = np.asarray(a.hist[:k + 1])
            with np.errstate(divide="ignore", invalid="ignore"):
                spread = np.maximum(spread, np.where(h > 0, np.abs(ha - h) / h,
                                                     np.where(ha == h, 0.0, np.inf)))
        # the sensitivity grows with j: a running maximum smooths the estimate,
        # and the residual norm is taken to be at least as sensitive as x_j
        spread = np.maximum.accumulate(spread)
        spread = np.maximum(spread, [self.spread_x(j) for j in range(k + 1)])
        bars = np.maximum(floor, SPREAD_FACTOR * spread)
        det = np.array([self.determined(j) for j in range(k + 1)])
        return np.where((bars <= DETERMINED) & det, bars, np.nan)

    def hist_ok(self, k, hist_gpu, floor):
        """GPU history within the bar wherever the entry is determined, judged
        against the nearest of the runs."""
        bars = self.hist_bars(k, floor)
        g = np.asarray(hist_gpu[:k + 1])
        best = np.full(k + 1, np.inf)
        for r in self.runs:
            h = np.asarray(r.hist[:k + 1])
            with np.errstate(divide="ignore", invalid="ignore"):
                d = np.where(h > 0, np.abs(g - h) / h, np.where(g == h, 0.0, np.inf))
            best = np.minimum(best, d)
        m = np.isfinite(bars)
        return bool(np.all(best[m] <= bars[m])), float(np.max(best[m] / bars[m], initial=0.0))


def oracle_spread(variant, A, b, d, k, **kw):
    """The oracle's x_k and the spread of x_k and of the history under two
    other rounding orders (see OracleBand)."""
    band = OracleBand(variant, A, b, d, k, **kw)
    ref = O.solve(variant, A, b, d=d, tol=0.0, maxit=k, **kw)
    h = np.asarray(ref.hist)
    sh = 0.0
    for a in band.alts:
        ha = np.asarray(a.hist)
        m = h > 0
        if np.any(m):
            sh = max(sh, float(np.max(np.abs(ha[m] - h[m]) / h[m])))
        if np.any(~m & (ha != h)):
            sh = np.inf
    return ref, band.spread_x(k), sh
