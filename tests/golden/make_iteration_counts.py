"""Write iteration_counts.txt: the oracle's iteration counts to 1e-10.

Calls only ``oracle/`` and the seeded generators in ``problems/``.  For each
benchmark system and variant it runs the oracle (Algorithms 1-3, the
stopping rule on the updated residual ||r_k|| / ||b||) from x_0 = 0 to a
relative residual of 1e-10 and records K, the number of completed
iterations, with the final updated and true relative residuals.  The GPU
tests hold the library's K to within 5 % of these counts.

    python tests/golden/make_iteration_counts.py [--jobs 4]

At 256^3 one oracle iteration takes about 0.3 s on one core, so the whole
table takes several minutes; each (system, variant, preconditioner) runs in
its own process.
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "iteration_counts.txt")

# (system tag, variant, preconditioner)
JOBS = [(sysname, v, pc)
        for sysname in ("poisson3d_256", "varcoef3d_128", "poisson2d_64")
        for pc in ("jacobi", "none")
        for v in ("pr", "hs", "pipe_pr")
        if not (sysname == "varcoef3d_128" and pc == "none")]
TOL = 1e-10


def _problem(sysname):
    import problems as P
    if sysname == "poisson3d_256":
        return P.poisson3d(256)
    if sysname == "varcoef3d_128":
        return P.varcoef3d(128)
    if sysname == "poisson2d_64":
        return P.poisson2d_64()
    raise KeyError(sysname)


def _run(job):
    sys.path.insert(0, ROOT)
    import numpy as np
    import scipy.sparse as sp
    import oracle as O
    sysname, variant, pc = job
    prob = _problem(sysname)
    rp, ci, v = prob.csr
    A = sp.csr_matrix((v, ci, rp), shape=(prob.n, prob.n))
    d = O.jacobi_inverse_diagonal(A) if pc == "jacobi" else None
    t0 = time.time()
    res = O.solve(variant, A, prob.b, d=d, tol=TOL, maxit=20 * prob.n if prob.n < 10**5 else 20000)
    tr = O.true_relres(A, prob.b, res.x)
    return (sysname, variant, pc, res.iters, res.status, res.hist[-1], tr, time.time() - t0,
            np.dtype(np.float64).name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=4)
    args = ap.parse_args()
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        rows = pool.map(_run, JOBS, chunksize=1)
    import platform
    with open(OUT, "w") as f:
        f.write("# Oracle iteration counts to ||r_K|| / ||b|| <= 1e-10 from x_0 = 0, written by\n")
        f.write("# make_iteration_counts.py (oracle/ and problems/ only; host %s).\n"
                % platform.machine())
        f.write("# Stopping rule on the updated residual; b = A x_true, x_true ~ U(-1, 1) seeded.\n")
        f.write("# system variant precond K status final_updated_relres final_true_relres\n")
        for sysname, variant, pc, k, st, h, tr, secs, _ in rows:
            f.write(f"{sysname} {variant} {pc} {k} {st} {h:.6e} {tr:.6e}\n")
            print(sysname, variant, pc, k, st, f"{h:.3e}", f"{tr:.3e}", f"{secs:.0f}s", flush=True)


if __name__ == "__main__":
    main()
