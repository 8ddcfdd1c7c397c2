"""Shared helpers of the GPU tests: problem cases and oracle-side matrices."""
import numpy as np
import scipy.sparse as sp

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
