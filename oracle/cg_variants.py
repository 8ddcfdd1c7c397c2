"""CPU oracle for the predict-and-recompute conjugate gradient variants.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.
The CUDA library never calls it and shares no code with it.

Every variant is written out step by step in the order and notation of
Chen & Carson, "Predict-and-recompute conjugate gradient variants":

* HS-CG     -- Algorithm 1 (Hestenes-Stiefel, preconditioned)
* PR-CG     -- Algorithm 2, with nu'_k from Eq. 2.3 and the four inner
               products of Eq. 2.4
* pipe-PR-CG-- Algorithm 3 (Section 2.2) with the recurrences for s, s~,
               w, w~ derived just before it
* M-CG, pipe-PR-M-CG, CG-CG, GV-CG -- the algorithms of Appendix E
* initialize() -- the initialisation algorithm of Appendix E, taken in
               dependency order (the printed listing repeats alpha_0 and
               s~_0 and lists w_0 before s~_0 is needed)

Arithmetic is whatever the array dtype gives: float64 numpy arrays for the
FP64 oracle, or object arrays of ``fractions.Fraction`` for exact rational
arithmetic (used by the tests to check that every variant reproduces
HS-CG's iterates exactly, Section 1: the variants are mathematically
equivalent).  A library matrix-vector product (numpy / scipy) is the only
primitive used; no blocking, fusion or reordering is done.

Readings where the paper is silent (shared with the GPU library):

* stopping: stop at the first k >= 0 with ||r_k|| / ||b|| <= tol, where
  ||r_k||^2 = <r_k, r_k> is the updated residual (one extra inner product
  when a preconditioner is used; equal to nu_k without one); x_k is
  returned;
* the scalars alpha_{k-1}, nu'_k, beta_k are formed at the start of
  iteration k (Section 2.2.1); if they are unusable (mu <= 0, nu <= 0,
  nu' < 0 or non-finite; Section 3.1: the methods break down when nu'
  turns negative, while nu' = 0 is the exact prediction of a zero residual)
  the run stops with status BREAKDOWN and returns x_{k-1} (K = k-1);
* the Jacobi preconditioner is M^{-1} = diag(d), d_i = 1 / a_ii, applied as
  an elementwise product inside the algorithm;
* sigma_k = <r~_k, s_k> (Eq. 2.3 / 2.4), not <s~_k, r_k>.
"""
from __future__ import annotations

import dataclasses
from fractions import Fraction
from typing import Callable, List, Optional

import numpy as np

OK = 0
NOT_CONVERGED = 1
BREAKDOWN = 2

VARIANTS = ("hs", "pr", "pipe_pr", "m", "pipe_m", "cgcg", "gv")


# ----------------------------------------------------------------------------
# primitives: matrix-vector product, preconditioner, inner product
# ----------------------------------------------------------------------------

def as_operator(A) -> Callable[[np.ndarray], np.ndarray]:
    """y = A v for a dense ndarray (float or Fraction), a scipy matrix or a callable."""
    if callable(A) and not hasattr(A, "shape"):
        return A
    if isinstance(A, np.ndarray):
        if A.dtype == object:
            return lambda v: A.dot(v)
        return lambda v: A @ v
    return lambda v: A @ v  # scipy.sparse


def jacobi_inverse_diagonal(A) -> np.ndarray:
    """d = 1 / diag(A) (Section 4: simple Jacobi preconditioner)."""
    if isinstance(A, np.ndarray):
        diag = np.array([A[i, i] for i in range(A.shape[0])], dtype=A.dtype)
    else:
        diag = np.asarray(A.diagonal(), dtype=np.float64)
    if diag.dtype == object:
        return np.array([Fraction(1) / v for v in diag], dtype=object)
    return 1.0 / diag


def _dot(a, b):
    return a.dot(b) if a.dtype == object else float(np.dot(a, b))


def _finite(v) -> bool:
    if isinstance(v, Fraction):
        return True
    return bool(np.isfinite(v))


def _sqrt(v):
    if isinstance(v, Fraction):
        return float(v) ** 0.5
    return float(np.sqrt(v)) if v >= 0 else float("nan")


@dataclasses.dataclass
class Result:
    """Outcome of one oracle run.

    x        -- x_K
    iters    -- K, the number of completed iterations
    status   -- OK / NOT_CONVERGED / BREAKDOWN
    hist     -- ||r_k|| / ||b|| for k = 0..K (updated residual)
    scalars  -- per completed iteration k >= 1 a dict of the scalars formed in
                it (alpha = alpha_{k-1}, beta = beta_k, nu = nu_k, mu = mu_k,
                sigma, gamma, nu_pred = nu'_k, eta); entry 0 is initialize()
    iterates -- (x_k, r_k) for k = 0..min(K, record) when record > 0
    extra    -- per-iteration diagnostics requested by ``track``
    """
    x: np.ndarray
    iters: int
    status: int
    hist: List[float]
    scalars: List[dict]
    iterates: List[tuple]
    extra: dict


class _Run:
    """Shared bookkeeping: stopping test, history, recorded iterates."""

    def __init__(self, A, b, x0, d, tol, maxit, record, track):
        self.A = as_operator(A)
        self.Amat = A
        self.b = b
        self.d = d
        self.tol = tol
        self.maxit = maxit
        self.record = record
        self.track = track or ()
        self.hist = []
        self.scalars = []
        self.iterates = []
        self.extra = {t: [] for t in self.track}
        self.bnorm = _sqrt(_dot(b, b))
        self.x0 = x0

    def Minv(self, v):
        return v if self.d is None else self.d * v

    def log(self, k, x, r, rho):
        """Record ||r_k||/||b||; return True when the stopping test holds."""
        # b == 0 counts as converged; a non-finite ||b|| stays non-finite, so
        # the test fails and the variant breaks down on its scalars
        rel = _sqrt(rho) / self.bnorm if self.bnorm != 0 else 0.0
        self.hist.append(rel)
        if self.record and k <= self.record:
            self.iterates.append((x.copy(), r.copy()))
        if isinstance(rho, Fraction):
            return rho == 0 or (self.tol > 0 and rel <= self.tol)
        return rel <= self.tol

    def result(self, x, k, status):
        return Result(x, k, status, self.hist, self.scalars, self.iterates, self.extra)


def _bad_alpha(nu, mu) -> bool:
    return (not _finite(nu)) or (not _finite(mu)) or mu <= 0 or nu < 0


def _start(A, b, x0, d, tol, maxit, record, track):
    n = b.shape[0]
    if x0 is None:
        x0 = np.zeros(n, dtype=b.dtype) if b.dtype != object else \
            np.array([Fraction(0)] * n, dtype=object)
    if maxit is None:
        maxit = 2 * n
    run = _Run(A, b, x0, d, tol, maxit, record, track)
    return run, x0.copy()


# ----------------------------------------------------------------------------
# initialize() (Appendix E), taken in dependency order
# ----------------------------------------------------------------------------

def initialize(run: _Run, x0, need_pipe: bool):
    A, Minv = run.A, run.Minv
    r = run.b - A(x0)                      # r_0 = b - A x_0
    rt = Minv(r)                           # r~_0 = M^{-1} r_0
    nu = _dot(r, rt)                       # nu_0 = <r_0, r~_0>
    p = rt.copy()                          # p_0 = r~_0
    s = A(p)                               # s_0 = A p_0
    mu = _dot(p, s)                        # <p_0, s_0>, alpha_0 = nu_0 / <p_0, s_0>
    st = Minv(s)                           # s~_0 = M^{-1} s_0
    sigma = _dot(rt, s)                    # sigma_0 = <r~_0, s_0>
    gamma = _dot(st, s)                    # gamma_0 = <s~_0, s_0>
    state = dict(r=r, rt=rt, nu=nu, p=p, s=s, mu=mu, st=st, sigma=sigma, gamma=gamma)
    if need_pipe:
        w = A(rt)                          # w_0 = A r~_0
        state.update(w=w, wt=Minv(w))      # w~_0 = M^{-1} w_0
        u = A(st)                          # u_0 = A s~_0
        state.update(u=u, ut=Minv(u))      # u~_0 = M^{-1} u_0
    rho = _dot(r, r)
    state["rho"] = rho
    run.scalars.append(dict(nu=nu, mu=mu, sigma=sigma, gamma=gamma, rho=rho))
    return state


def _gap_tracks(run, k, x, r, st=None, w=None):
    """Record tracked quantities; `st` is a callable, evaluated only when the
    nu'-gap is tracked (its <r, r> is not part of the iteration's work)."""
    if "nu_gap" in run.track and st is not None:
        run.extra["nu_gap"].append((k, st()))
    if "w_gap" in run.track and w is not None:
        run.extra["w_gap"].append((k, w))


# ----------------------------------------------------------------------------
# Algorithm 1: HS-CG
# ----------------------------------------------------------------------------

def hs_cg(A, b, x0=None, d=None, tol=0.0, maxit=None, record=0, track=None):
    run, x = _start(A, b, x0, d, tol, maxit, record, track)
    I = initialize(run, x, need_pipe=False)
    r, p, s, nu, mu = I["r"], I["p"], I["s"], I["nu"], I["mu"]
    if run.log(0, x, r, I["rho"]):
        return run.result(x, 0, OK)
    if run.bnorm == 0:
        return run.result(x, 0, OK)
    for k in range(1, run.maxit + 1):
        if _bad_alpha(nu, mu):
            return run.result(x, k - 1, BREAKDOWN)
        alpha = nu / mu                      # alpha_{k-1} = nu_{k-1} / mu_{k-1}
        x = x + alpha * p                    # x_k = x_{k-1} + alpha_{k-1} p_{k-1}
        r = r - alpha * s                    # r_k = r_{k-1} - alpha_{k-1} s_{k-1}
        rt = run.Minv(r)                     # r~_k = M^{-1} r_k
        nu_new = _dot(rt, r)                 # nu_k = <r~_k, r_k>
        rho = nu_new if run.d is None else _dot(r, r)
        sc = dict(alpha=alpha, nu=nu_new, rho=rho)
        run.scalars.append(sc)
        if run.log(k, x, r, rho):
            return run.result(x, k, OK)
        if (not _finite(nu_new)) or nu_new <= 0:
            return run.result(x, k, BREAKDOWN)
        beta = nu_new / nu                   # beta_k = nu_k / nu_{k-1}
        p = rt + beta * p                    # p_k = r~_k + beta_k p_{k-1}
        s = run.A(p)                         # s_k = A p_k
        mu = _dot(p, s)                      # mu_k = <p_k, s_k>
        nu = nu_new
        sc.update(beta=beta, mu=mu)
        _gap_tracks(run, k, x, r)
    return run.result(x, run.maxit, NOT_CONVERGED)


# ----------------------------------------------------------------------------
# Algorithm 2: PR-CG (and M-CG, Appendix E, which differs only in nu'_k)
# ----------------------------------------------------------------------------

def pr_cg(A, b, x0=None, d=None, tol=0.0, maxit=None, record=0, track=None,
          meurant=False, recompute_nu=True):
    """PR-CG (Alg. 2); ``meurant`` gives M-CG; ``recompute_nu=False`` is the
    ablation of Eq. 3.17 where nu'_k is carried from nu'_{k-1} and the inner
    product nu_k is never used (Fig. 1)."""
    run, x = _start(A, b, x0, d, tol, maxit, record, track)
    I = initialize(run, x, need_pipe=False)
    r, rt, p, s, st = I["r"], I["rt"], I["p"], I["s"], I["st"]
    nu, mu, sigma, gamma = I["nu"], I["mu"], I["sigma"], I["gamma"]
    if run.log(0, x, r, I["rho"]):
        return run.result(x, 0, OK)
    if run.bnorm == 0:
        return run.result(x, 0, OK)
    for k in range(1, run.maxit + 1):
        # scalar step at the start of the iteration (Section 2.2.1)
        if _bad_alpha(nu, mu):
            return run.result(x, k - 1, BREAKDOWN)
        alpha = nu / mu                                            # alpha_{k-1}
        if meurant:
            nu_pred = -nu + alpha * alpha * gamma                  # M-CG
        else:
            nu_pred = nu - 2 * alpha * sigma + alpha * alpha * gamma  # Eq. 2.3
        if (not _finite(nu_pred)) or nu_pred < 0 or nu == 0:
            return run.result(x, k - 1, BREAKDOWN)
        beta = nu_pred / nu                                        # beta_k = nu'_k / nu_{k-1}
        # vector updates
        x = x + alpha * p                                          # x_k
        r = r - alpha * s                                          # r_k
        rt = r if run.d is None else rt - alpha * st               # r~_k by recurrence
        p = rt + beta * p                                          # p_k
        s = run.A(p)                                               # s_k = A p_k
        st = run.Minv(s)                                           # s~_k = M^{-1} s_k
        # the inner products, all in one reduction
        mu = _dot(p, s)                                            # mu_k
        if not meurant:   # Meurant's nu' (Appendix E) reads no sigma
            sigma = _dot(rt, s)                                        # sigma_k
        gamma = _dot(st, s)                                        # gamma_k
        nu_true = _dot(rt, r)                                      # nu_k (recomputed)
        rho = nu_true if run.d is None else _dot(r, r)
        nu = nu_true if recompute_nu else nu_pred
        run.scalars.append(dict(alpha=alpha, beta=beta, nu_pred=nu_pred, nu=nu_true,
                                mu=mu, sigma=sigma, gamma=gamma, rho=rho))
        if meurant:
            del run.scalars[-1]["sigma"]
        _gap_tracks(run, k, x, r, st=lambda: (nu_pred, _dot(r, r)))
        if run.log(k, x, r, rho):
            return run.result(x, k, OK)
    return run.result(x, run.maxit, NOT_CONVERGED)


def m_cg(A, b, **kw):
    """M-CG (Appendix E): PR-CG with nu'_k = -nu_{k-1} + alpha_{k-1}^2 gamma_{k-1}."""
    return pr_cg(A, b, meurant=True, **kw)


# ----------------------------------------------------------------------------
# Algorithm 3: pipe-PR-CG (and pipe-PR-M-CG, Appendix E)
# ----------------------------------------------------------------------------

def pipe_pr_cg(A, b, x0=None, d=None, tol=0.0, maxit=None, record=0, track=None,
               meurant=False, recompute_w=True):
    """pipe-PR-CG (Alg. 3); ``meurant`` gives pipe-PR-M-CG; ``recompute_w=False``
    is the ablation where w_k = w'_k is never recomputed (Fig. 2)."""
    run, x = _start(A, b, x0, d, tol, maxit, record, track)
    I = initialize(run, x, need_pipe=True)
    r, rt, p, s, st = I["r"], I["rt"], I["p"], I["s"], I["st"]
    w, wt, u, ut = I["w"], I["wt"], I["u"], I["ut"]
    nu, mu, sigma, gamma = I["nu"], I["mu"], I["sigma"], I["gamma"]
    pc = run.d is not None
    if run.log(0, x, r, I["rho"]):
        return run.result(x, 0, OK)
    if run.bnorm == 0:
        return run.result(x, 0, OK)
    for k in range(1, run.maxit + 1):
        if _bad_alpha(nu, mu):
            return run.result(x, k - 1, BREAKDOWN)
        alpha = nu / mu                                            # alpha_{k-1}
        if meurant:
            nu_pred = -nu + alpha * alpha * gamma
        else:
            nu_pred = nu - 2 * alpha * sigma + alpha * alpha * gamma
        if (not _finite(nu_pred)) or nu_pred < 0 or nu == 0:
            return run.result(x, k - 1, BREAKDOWN)
        beta = nu_pred / nu                                        # beta_k
        x = x + alpha * p                                          # x_k
        r = r - alpha * s                                          # r_k
        rt = rt - alpha * st if pc else r                          # r~_k
        wp = w - alpha * u                                         # w'_k
        wtp = wt - alpha * ut if pc else wp                        # w~'_k
        p = rt + beta * p                                          # p_k
        s = wp + beta * s                                          # s_k = w'_k + beta_k s_{k-1}
        st = wtp + beta * st if pc else s                          # s~_k
        u = run.A(st)                                              # u_k = A s~_k
        ut = run.Minv(u)                                           # u~_k = M^{-1} u_k
        if recompute_w:
            w = run.A(rt)                                          # w_k = A r~_k (recomputed)
            wt = run.Minv(w)                                       # w~_k = M^{-1} w_k
        else:
            w, wt = wp, wtp
        mu = _dot(p, s)
        if not meurant:   # Meurant's nu' (Appendix E) reads no sigma
            sigma = _dot(rt, s)
        gamma = _dot(st, s)
        nu_true = _dot(rt, r)
        rho = nu_true if not pc else _dot(r, r)
        nu = nu_true
        run.scalars.append(dict(alpha=alpha, beta=beta, nu_pred=nu_pred, nu=nu_true,
                                mu=mu, sigma=sigma, gamma=gamma, rho=rho))
        if meurant:
            del run.scalars[-1]["sigma"]
        _gap_tracks(run, k, x, r, st=lambda: (nu_pred, _dot(r, r)), w=(r, wp))
        if run.log(k, x, r, rho):
            return run.result(x, k, OK)
    return run.result(x, run.maxit, NOT_CONVERGED)


def pipe_m_cg(A, b, **kw):
    """pipe-PR-M-CG (Appendix E)."""
    return pipe_pr_cg(A, b, meurant=True, **kw)


# ----------------------------------------------------------------------------
# Appendix E: CG-CG (Chronopoulos-Gear) and GV-CG (Ghysels-Vanroose)
# ----------------------------------------------------------------------------

def cg_cg(A, b, x0=None, d=None, tol=0.0, maxit=None, record=0, track=None):
    run, x = _start(A, b, x0, d, tol, maxit, record, track)
    I = initialize(run, x, need_pipe=False)
    r, p, s, nu, mu = I["r"], I["p"], I["s"], I["nu"], I["mu"]
    if run.log(0, x, r, I["rho"]):
        return run.result(x, 0, OK)
    if run.bnorm == 0:
        return run.result(x, 0, OK)
    if _bad_alpha(nu, mu):
        return run.result(x, 0, BREAKDOWN)
    alpha = nu / mu                                                # alpha_0
    for k in range(1, run.maxit + 1):
        x = x + alpha * p
        r = r - alpha * s
        rt = run.Minv(r)                                           # r~_k = M^{-1} r_k
        w = run.A(rt)                                              # w_k = A r~_k
        nu_new = _dot(rt, r)                                       # nu_k
        eta = _dot(rt, w)                                          # eta_k
        rho = nu_new if run.d is None else _dot(r, r)
        sc = dict(alpha=alpha, nu=nu_new, eta=eta, rho=rho)
        run.scalars.append(sc)
        if run.log(k, x, r, rho):
            return run.result(x, k, OK)
        if (not _finite(nu_new)) or nu_new <= 0:
            return run.result(x, k, BREAKDOWN)
        beta = nu_new / nu                                         # beta_k
        p = rt + beta * p
        s = w + beta * s
        mu = eta - (beta / alpha) * nu_new                         # mu_k
        if _bad_alpha(nu_new, mu):
            return run.result(x, k, BREAKDOWN)
        alpha = nu_new / mu                                        # alpha_k
        nu = nu_new
        sc.update(beta=beta, mu=mu)
    return run.result(x, run.maxit, NOT_CONVERGED)


def gv_cg(A, b, x0=None, d=None, tol=0.0, maxit=None, record=0, track=None):
    run, x = _start(A, b, x0, d, tol, maxit, record, track)
    I = initialize(run, x, need_pipe=True)
    r, rt, p, s, st = I["r"], I["rt"], I["p"], I["s"], I["st"]
    w, u = I["w"], I["u"]
    nu, mu = I["nu"], I["mu"]
    pc = run.d is not None
    if run.log(0, x, r, I["rho"]):
        return run.result(x, 0, OK)
    if run.bnorm == 0:
        return run.result(x, 0, OK)
    if _bad_alpha(nu, mu):
        return run.result(x, 0, BREAKDOWN)
    alpha = nu / mu
    for k in range(1, run.maxit + 1):
        x = x + alpha * p
        r = r - alpha * s
        rt = rt - alpha * st if pc else r                          # r~_k by recurrence
        w = w - alpha * u                                          # w_k by recurrence
        wt = run.Minv(w)                                           # w~_k = M^{-1} w_k
        nu_new = _dot(rt, r)
        eta = _dot(rt, w)
        rho = nu_new if not pc else _dot(r, r)
        sc = dict(alpha=alpha, nu=nu_new, eta=eta, rho=rho)
        run.scalars.append(sc)
        if run.log(k, x, r, rho):
            return run.result(x, k, OK)
        t = run.A(wt)                                              # t_k = A w~_k
        if (not _finite(nu_new)) or nu_new <= 0:
            return run.result(x, k, BREAKDOWN)
        beta = nu_new / nu
        p = rt + beta * p
        s = w + beta * s
        st = wt + beta * st if pc else s
        u = t + beta * u
        mu = eta - (beta / alpha) * nu_new
        if _bad_alpha(nu_new, mu):
            return run.result(x, k, BREAKDOWN)
        alpha = nu_new / mu
        nu = nu_new
        sc.update(beta=beta, mu=mu)
    return run.result(x, run.maxit, NOT_CONVERGED)


SOLVERS = {
    "hs": hs_cg,
    "pr": pr_cg,
    "pipe_pr": pipe_pr_cg,
    "m": m_cg,
    "pipe_m": pipe_m_cg,
    "cgcg": cg_cg,
    "gv": gv_cg,
}


def solve(variant: str, A, b, **kw) -> Result:
    """Run one variant by name (see ``VARIANTS``)."""
    return SOLVERS[variant](A, b, **kw)


def true_relres(A, b, x) -> float:
    """||b - A x|| / ||b|| with the library matrix-vector product."""
    r = b - as_operator(A)(x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def a_norm_error(A, x_star, x) -> float:
    """||x* - x||_A."""
    e = x_star - x
    return float(np.sqrt(max(_dot(e, as_operator(A)(e)), 0.0)))
