"""The parity bar itself can fail (CPU; no GPU).

gpu_common.OracleBand sets the element-wise bar of the GPU parity tests: 1e-10
where the iterates are determined by FP64 arithmetic, else 8 x the oracle's
spread over three other roundings, never above 1e-6.  Here a stand-in
for the GPU -- the oracle under yet another rounding order (per-lane strided
inner products, every product summed in reverse) -- must pass that bar on
every case, and copies of the oracle with a planted mistake must fail it on
the ill-conditioned unpreconditioned sigma = 2 diffusion case, including
mistakes that appear only after several iterations or change a scalar by a
relative 1e-8.
"""
import os
import sys
import types

import numpy as np
import pytest

import oracle as O
import oracle.cg_variants as CV
from gpu_common import CASES, DETERMINED, OracleBand, _reversed_rows, case, csr_matrix

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "cg_variants.py")
KS = (1, 2, 7, 10, 15, 20)


def _lane_dot(u, v):
    """Inner product as 32 strided lane partials added in reverse lane order."""
    if u.dtype == object:
        return u.dot(v)
    p = u * v
    m = (len(p) + 31) // 32 * 32
    q = np.zeros(m)
    q[:len(p)] = p
    return float(np.sum(q.reshape(-1, 32).sum(axis=0)[::-1]))


def _stand_in(mod, variant, A, b, d):
    Ar = _reversed_rows(A)
    saved = mod._dot
    mod._dot = _lane_dot
    try:
        return mod.solve(variant, lambda v: Ar @ v, b, d=d, tol=0.0, maxit=KS[-1], record=KS[-1])
    finally:
        mod._dot = saved


def _passes(band, run):
    for k in KS:
        if band.determined(k) and band.dist_x(k, run.iterates[k][0]) > band.bar_x(k):
            return False
        ok, _ = band.hist_ok(k, run.hist, 1e-9)
        if not ok:
            return False
    return True


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precond", ["none", "jacobi"])
def test_another_rounding_order_passes(name, precond):
    prob = case(name)
    A = csr_matrix(prob)
    d = O.jacobi_inverse_diagonal(A) if precond == "jacobi" else None
    for variant in ("hs", "pr", "pipe_pr", "gv"):
        band = OracleBand(variant, A, prob.b, d, KS[-1])
        assert _passes(band, _stand_in(CV, variant, A, prob.b, d)), (name, precond, variant)
        # every case is compared element by element at least up to k = 10
        assert all(band.determined(k) for k in KS if k <= 10)
        assert all(band.bar_x(k) <= DETERMINED for k in KS if band.determined(k))


def _mutant(old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, old
    name = "oracle_bar_mutant_%d" % abs(hash((old, new)))
    mod = types.ModuleType(name)
    sys.modules[name] = mod
    exec(compile(src.replace(old, new), name, "exec"), mod.__dict__)
    return mod


MUTATIONS = {
    # Eq. 2.3 with the alpha^2 gamma term perturbed by a relative 1e-8
    "nu_pred_1e-8": ("pr", "nu_pred = nu - 2 * alpha * sigma + alpha * alpha * gamma  # Eq. 2.3",
                     "nu_pred = nu - 2 * alpha * sigma + alpha * alpha * gamma * (1 + 1e-8)"),
    # the p update wrong from iteration 8 on only
    "late_p_update": ("pr", "p = rt + beta * p                                          # p_k",
                      "p = rt + beta * p if k < 8 else rt + beta * p * (1 + 1e-9)"),
    # sigma_k off by a relative 1e-7
    "sigma_1e-7": ("pipe_pr", "sigma = _dot(rt, s)", "sigma = _dot(rt, s) * (1 - 1e-7)"),
    # x update skipped once at iteration 12
    "x_skip_12": ("hs", "x = x + alpha * p                    # x_k = x_{k-1} + alpha_{k-1} p_{k-1}",
                  "x = x + alpha * p if k != 12 else x"),
    # GV-CG's w recurrence off by a relative 1e-9 in its step from k = 5 on
    "gv_w_late": ("gv", "w = w - alpha * u                                          # w_k by recurrence",
                  "w = w - alpha * u if k < 5 else w - alpha * u * (1 + 1e-9)"),
}


@pytest.mark.parametrize("mut", list(MUTATIONS))
def test_planted_mistakes_fail_on_the_ill_conditioned_case(mut):
    variant, old, new = MUTATIONS[mut]
    mod = _mutant(old, new)
    prob = case("varcoef2d_ragged")
    A = csr_matrix(prob)
    band = OracleBand(variant, A, prob.b, None, KS[-1])
    run = mod.solve(variant, A, prob.b, tol=0.0, maxit=KS[-1], record=KS[-1])
    assert not _passes(band, run), mut
