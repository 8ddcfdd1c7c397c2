"""The oracle-written iteration counts (tests/golden/iteration_counts.txt).

The GPU tests hold the library's iteration count to 1e-10 within 5 % of
these.  Here, without a GPU: the file covers every system the GPU tests read,
every run converged with a true residual at the tolerance, the variants agree
with each other (they are mathematically equivalent, Section 1, so their
counts differ only through rounding), and the small 2D entry is reproduced
by running the oracle again.
"""
import os

import pytest
import scipy.sparse as sp

import oracle as O
import problems as P

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "iteration_counts.txt")


def _rows():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out[(line[0], line[1], line[2])] = (int(line[3]), int(line[4]), float(line[5]),
                                                    float(line[6]))
    return out


def test_golden_counts_cover_the_benchmark_systems():
    rows = _rows()
    for system, pcs in (("poisson3d_256", ("jacobi", "none")), ("varcoef3d_128", ("jacobi",)),
                        ("poisson2d_64", ("jacobi", "none"))):
        for pc in pcs:
            ks = []
            for v in ("pr", "hs", "pipe_pr"):
                k, status, upd, true = rows[(system, v, pc)]
                assert status == O.OK and upd <= 1e-10 and true <= 1e-9, (system, v, pc)
                ks.append(k)
            assert max(ks) - min(ks) <= 0.05 * min(ks), (system, pc, ks)


@pytest.mark.parametrize("variant", ["pr", "hs", "pipe_pr"])
def test_golden_count_reproduced_on_poisson2d_64(variant):
    prob = P.poisson2d_64()
    rp, ci, v = prob.csr
    A = sp.csr_matrix((v, ci, rp), shape=(prob.n, prob.n))
    res = O.solve(variant, A, prob.b, tol=1e-10, maxit=2 * prob.n)
    k = _rows()[("poisson2d_64", variant, "none")][0]
    assert abs(res.iters - k) <= 1, (res.iters, k)
