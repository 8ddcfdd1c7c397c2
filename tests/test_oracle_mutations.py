"""Plant plausible mistakes in a copy of the oracle and check that a pin fails.

Each mutation is a textual edit of oracle/cg_variants.py (a dropped term, a
flipped sign, a wrong operand or a skipped recompute) executed as a separate
module; the real oracle is untouched.
"""
import os
import sys
import types
import numpy as np
import pytest

import problems as P

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "cg_variants.py")
EPS = 2.0 ** -53


def _load(old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, old
    name = "oracle_mutant_%d" % abs(hash((old, new)))
    mod = types.ModuleType(name)
    sys.modules[name] = mod
    exec(compile(src.replace(old, new), name, "exec"), mod.__dict__)
    return mod


def _exact_pin_fails(O, variant, precond=False):
    rng = np.random.default_rng(3)
    A = P.random_int_spd(6, rng)
    b = P.fraction_vector(rng.integers(-5, 6, size=6))
    d = O.jacobi_inverse_diagonal(A) if precond else None
    ref = O.hs_cg(A, b, d=d, record=8, maxit=7)
    try:
        res = O.solve(variant, A, b, d=d, record=8, maxit=7)
    except Exception:
        return True
    if res.iters != ref.iters or res.status != O.OK:
        return True
    return any(not (all(xa == xb) and all(ra == rb))
               for (xa, ra), (xb, rb) in zip(ref.iterates, res.iterates))


def _termination_pin_fails(O, variant):
    rng = np.random.default_rng(1)
    A = P.int_spd_with_eigs([1, 1, 2, 3, 3, 5], rng)
    b = P.fraction_vector([1, 2, 3, 1, 2, 3])
    try:
        res = O.solve(variant, A, b, maxit=5)
    except Exception:
        return True
    return res.status != O.OK or res.iters > 4 or not all(A.dot(res.x) == b)


def _w_gap_pin_fails(O):
    prob = P.model_problem(48, 0.8, 1e3)
    res = O.pipe_pr_cg(prob.A, prob.b, maxit=120, track=("w_gap",))
    An = np.linalg.norm(prob.A, 2)
    c = 48 * np.sqrt(48)
    prev = None
    for _, (rk, wp) in res.extra["w_gap"]:
        nr = np.linalg.norm(rk)
        prev = nr if prev is None else prev
        if np.linalg.norm(prob.A @ rk - wp) > EPS * c * An * (nr + prev):
            return True
        prev = nr
    return False


def _accuracy_pin_fails(O, variant):
    prob = P.model_problem(48, 0.8, 1e3)
    res = O.solve(variant, prob.A, prob.b, maxit=300)
    return min(res.hist) > 1e-12


MUTATIONS = [
    # (variant checked, old text, new text, pin)
    ("pr", "nu - 2 * alpha * sigma + alpha * alpha * gamma  # Eq. 2.3",
     "nu + 2 * alpha * sigma + alpha * alpha * gamma  # Eq. 2.3", "exact"),
    ("pr", "nu - 2 * alpha * sigma + alpha * alpha * gamma  # Eq. 2.3",
     "nu - 2 * alpha * sigma  # Eq. 2.3", "exact"),
    ("pr", "sigma = _dot(rt, s)                                        # sigma_k",
     "sigma = _dot(rt, r)                                        # sigma_k", "exact"),
    ("pr", "gamma = _dot(st, s)                                        # gamma_k",
     "gamma = _dot(st, st)                                       # gamma_k", "exact_pc"),
    ("pipe_pr", "s = wp + beta * s                                          # s_k",
     "s = wp - beta * s                                          # s_k", "exact"),
    ("pipe_pr", "wp = w - alpha * u                                         # w'_k",
     "wp = w - alpha * s                                         # w'_k", "exact"),
    ("pipe_pr", "st = wtp + beta * st if pc else s                          # s~_k",
     "st = wtp + beta * p if pc else s                           # s~_k", "exact_pc"),
    ("pipe_pr", "if recompute_w:", "if False:", "w_gap"),
    ("pr", "nu = nu_true if recompute_nu else nu_pred", "nu = nu_pred", "accuracy"),
    ("hs", "r = r - alpha * s                    # r_k = r_{k-1} - alpha_{k-1} s_{k-1}",
     "r = r - alpha * p                    # r_k = r_{k-1} - alpha_{k-1} s_{k-1}", "termination"),
    ("hs", "beta = nu_new / nu                   # beta_k = nu_k / nu_{k-1}",
     "beta = nu / nu_new                   # beta_k = nu_k / nu_{k-1}", "termination"),
    ("pr", "mu = _dot(p, s)                        # <p_0, s_0>",
     "mu = _dot(p, p)                        # <p_0, s_0>", "exact"),
    ("gv", "u = t + beta * u", "u = t + beta * s", "exact"),
    ("cgcg", "mu = eta - (beta / alpha) * nu_new                         # mu_k",
     "mu = eta + (beta / alpha) * nu_new                         # mu_k", "exact"),
    ("m", "nu_pred = -nu + alpha * alpha * gamma                  # M-CG",
     "nu_pred = nu + alpha * alpha * gamma                   # M-CG", "exact"),
]


@pytest.mark.parametrize("variant,old,new,pin", MUTATIONS)
def test_pin_catches_mutation(variant, old, new, pin):
    O = _load(old, new)
    if pin == "exact":
        assert _exact_pin_fails(O, variant) or _exact_pin_fails(O, variant, True)
    elif pin == "exact_pc":
        assert _exact_pin_fails(O, variant, True)
    elif pin == "termination":
        assert _termination_pin_fails(O, variant)
    elif pin == "w_gap":
        assert _w_gap_pin_fails(O)
    elif pin == "accuracy":
        assert _accuracy_pin_fails(O, variant)


def test_unmutated_oracle_passes_the_same_pins():
    O = _load("", "")
    for v in ("hs", "pr", "pipe_pr", "m", "cgcg", "gv"):
        assert not _exact_pin_fails(O, v) and not _exact_pin_fails(O, v, True)
        assert not _termination_pin_fails(O, v)
    assert not _w_gap_pin_fails(O)
    assert not _accuracy_pin_fails(O, "pr")
