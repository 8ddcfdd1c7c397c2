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
    if name == "poisson3d_nx24":
        # nx a multiple of 4: the FP32 stencil product takes four rows at a time
        return P.grid_problem((24, 13, 11), "t_p3x")
    raise KeyError(name)


CASES = ["poisson2d_64", "poisson3d_ragged", "varcoef3d_ragged", "varcoef2d_ragged", "shifted2d"]
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


def oracle_spread(variant, A, b, d, k, **kw):
    """Rounding sensitivity of the iterates themselves: the oracle against the
    same oracle with exactly rounded inner products (math.fsum).  On
    ill-conditioned systems (unpreconditioned log-normal diffusion, sigma = 2)
    a change of summation order alone moves x_20 by up to ~1e-3, so no FP64
    implementation can match another to 1e-10 there; the bar becomes
    max(1e-10, 100 x this spread)."""
    import oracle.cg_variants as CV
    ref = O.solve(variant, A, b, d=d, tol=0.0, maxit=k, **kw)
    saved = CV._dot
    CV._dot = lambda u, v: saved(u, v) if u.dtype == object else _fsum_dot(u, v)
    try:
        alt = O.solve(variant, A, b, d=d, tol=0.0, maxit=k, **kw)
    finally:
        CV._dot = saved
    hs = np.asarray(ref.hist)
    return ref, rel(alt.x, ref.x), np.max(np.abs(np.asarray(alt.hist) - hs) / hs)
