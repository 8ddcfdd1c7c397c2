#!/usr/bin/env python
"""Benchmark: PR-CG vs HS-CG iterations/s and HBM GB/s on one GB300.

Default workload (the 3D configuration of the method's targets): 3D 7-point
Poisson on a 256^3 grid (n = 16,777,216, nnz = 117,047,296), FP64, CSR,
Jacobi preconditioner, x_true ~ U(-1, 1), b = A x_true, x_0 = 0, solved by
PR-CG to ||r_k|| / ||b|| <= 1e-10.  One step = one complete solve
(initialisation, iterations, device-side loop control) on resident inputs;
value = iterations / device time.  HS-CG, pipe-PR-CG, the matrix-free
stencil and the 128^3 log-normal diffusion system are reported beside it.

--impl reference times the CPU oracle (the multi-threaded C oracle on every
host core) on a bounded sample of the same workload.
"""
from __future__ import annotations

import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CG iters/s & HBM GB/s (PR vs HS-CG, FP64, 256^3); batched solves/s @1e-8"
L2_BYTES = 129e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------- models
def model_bytes(variant: str, op: str, precond: str, n: int, nnz: int, dim: int = 3,
                dvec=None) -> float:
    """Algorithmic DRAM bytes of one iteration, the fully fused minimum of the
    method (every vector read and written once per iteration, A read once).

    V = 8n bytes per vector sweep.  A = 12 nnz + 4 (n+1) for CSR, 0 for the
    constant stencil, ~(dim + 1) V for the variable-coefficient stencil (face
    arrays + diagonal).
      HS:   R x p r s, W x r; R r p, W p s (+A)       -> 10V + A
      PR:   R x p r s, W x r p s (+A)                  ->  8V + A
      pipe: R x p r s w u, W x r p s w u (+A)          -> 12V + A
    Jacobi adds r~ (PR, pipe) and s~ (pipe) read+write, and one read of d per
    sweep when d is a vector (CSR, variable coefficients).
    """
    V = 8.0 * n
    if op == "csr":
        A = 12.0 * nnz + 4.0 * (n + 1)
    elif op == "varcoef":
        A = (dim + 1) * V
    else:
        A = 0.0
    if dvec is None:
        dvec = precond == "jacobi" and op in ("csr", "varcoef")
    jac = precond == "jacobi"
    if variant == "hs":
        return 10 * V + A + (2 * V if dvec else 0.0)
    if variant in ("pr", "m"):
        return 8 * V + A + (2 * V if jac else 0.0) + (V if dvec else 0.0)
    if variant in ("pipe_pr", "pipe_m"):
        return 12 * V + A + (4 * V if jac else 0.0) + (V if dvec else 0.0)
    raise KeyError(variant)


def sweep_models(variant: str, op: str, precond: str, n: int, nnz: int, dvec=None,
                 int_row=False):
    """Per sweep of this library's schedule: (name, DRAM bytes the sweep must
    move, FP64 instructions it must execute), counted per row and x n.

    FP64 instructions are those this library issues for the algorithm (one
    FMA per stored matrix entry, one FMA per vector update and per
    inner-product term, one multiply per use of an explicit M^{-1} v).  A
    constant-coefficient stencil row counts 1: its neighbour sum is formed in
    fixed point on the integer pipes, leaving the FMA c p_i - sum; with
    `int_row` (an integer diagonal) the product sweeps form their rows from
    block fixed-point copies in integers and it counts 0.  Integer work and
    the copies' bytes are not counted (the bytes are the algorithm's).
    """
    V = 8.0 * n
    A = 12.0 * nnz + 4.0 * (n + 1) if op == "csr" else 0.0
    m = float(nnz) if op == "csr" else 1.0 * n
    # an integer stencil diagonal: the product sweeps, which read block
    # fixed-point copies, form their rows without an FP64 instruction
    m1 = 0.0 if (int_row and op == "stencil") else m
    if dvec is None:
        dvec = precond == "jacobi" and op == "csr"
    dv = 1.0 if dvec else 0.0   # read of vector d
    jac = precond == "jacobi"
    if variant == "hs":
        return [("k_hs_a", (6 + dv) * V, (5 if jac and dv else 3) * n),
                ("k_hs_b", (3 + dv) * V, (2 if jac else 1) * n),
                ("k_hs_c", 2 * V + A, m1 + n)]
    # a constant d is a scalar: r~ -= (alpha d) s is one FMA (a vector d forms
    # d s first); pipe-PR's w~' = d w' is one multiply for either form of d
    if variant in ("pr", "m"):
        if jac:
            return [("k_pr_a", (9 + dv) * V, (7 if dv else 6) * n),
                    ("k_pr_b", (3 + dv) * V + A, m1 + (4 if dv else 3) * n)]
        return [("k_pr_a", 7 * V, 4 * n), ("k_pr_b", 3 * V + A, m1 + 3 * n)]
    if variant in ("pipe_pr", "pipe_m"):
        if jac:
            return [("k_pipe", (12 + dv) * V + A, 2 * m1 + 13 * n)]
        return [("k_pipe", 8 * V + A, 2 * m1 + 9 * n)]
    raise KeyError(variant)


FP64_PER_SM_CLK = 2.0   # DFMA issue rate of a GB300 SM (ncu: sm__sass_thread_inst_executed_op_dfma peak)
N_SMS = 152


def fp64_peak(sm_mhz=None) -> float:
    """FP64 instructions/s of the whole GPU at the given (or maximum) SM clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mx = float(json.load(f).get("sm_max_mhz", 2070.0))
    except Exception:
        mx = 2070.0
    clk = sm_mhz if sm_mhz else mx
    return FP64_PER_SM_CLK * N_SMS * clk * 1e6


def sweep_roofline(S, variant, op, precond, n, nnz, reps=20, sm_mhz=None):
    """Time every sweep of one iteration with CUDA events (prcg_time_sweeps)
    and place the slowest one on both rooflines (HBM bytes, FP64 issue)."""
    from paper_1905_01549_gb300 import binding
    ms = binding.prcg_time_sweeps(S.handle, binding.VARIANT_IDS[variant], reps)
    models = sweep_models(variant, op, precond, n, nnz, dvec=S.jacobi_form == "vector",
                          int_row=S.int_diagonal > 0)
    peak_hbm, hbm_src = _peaks()
    peak_fp = fp64_peak(sm_mhz)
    per = []
    for (name, by, fp), t in zip(models, ms):
        ts = t / 1e3
        per.append({"kernel": name, "us": t * 1e3, "model_bytes": by, "model_fp64": fp,
                    "hbm_frac": by / ts / 1e9 / peak_hbm, "alu_frac": fp / ts / peak_fp})
    dom = max(range(len(per)), key=lambda q: per[q]["us"])
    d = per[dom]
    t_hbm = d["model_bytes"] / (peak_hbm * 1e9)
    t_alu = d["model_fp64"] / peak_fp
    if t_alu > t_hbm:
        roof = {"bound": "alu", "achieved": d["model_fp64"] / (d["us"] / 1e6) / 1e9,
                "peak": peak_fp / 1e9, "unit": "G FP64-inst/s", "frac": d["alu_frac"],
                "peak_source": "derived: 2 FP64 inst/clk/SM x 152 SMs x SM clock"}
    else:
        roof = {"bound": "hbm", "achieved": d["model_bytes"] / (d["us"] / 1e6) / 1e9,
                "peak": peak_hbm, "unit": "GB/s", "frac": d["hbm_frac"], "peak_source": hbm_src}
    roof.update({"kernel": d["kernel"], "launch_us": d["us"], "bytes_per_launch": d["model_bytes"],
                 "fp64_per_launch": d["model_fp64"], "hbm_frac": d["hbm_frac"],
                 "alu_frac": d["alu_frac"], "sweeps": per})
    return roof


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            why = ("nvidia-smi unavailable" if self.proc is None else
                   "no sample: the timed region ended before nvidia-smi's first reading")
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [why], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags)
                          if f.lower() in ("active", "1")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- workloads
def build_problem(name: str):
    import problems as P
    if name.startswith("poisson3d_"):
        return P.poisson3d(int(name.split("_")[1]))
    if name.startswith("varcoef3d_128"):
        return P.varcoef3d(128)
    raise KeyError(name)


def make_solver(G, prob, op, precond):
    if op == "csr":
        rp, ci, v = prob.csr
        return G.Solver.from_csr(rp, ci, v, precond=precond)
    return G.Solver.from_stencil(prob.dims, face_coeff=prob.face_array(), diag_shift=prob.shift,
                                 precond=precond)


# Sources that define the TMA-staged SELL product sweep and its launch
# configuration (the kernel whose DRAM traffic profiles/traffic.json records).
SWEEP_SOURCES = ("prcg_common.cuh", "prcg_reduce.cuh", "prcg_ops.cuh", "prcg_isum.cuh",
                 "prcg_tma.cuh", "prcg_launch.cuh", "prcg_inst_csr.cu", "prcg_inst_csr_sc.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1905_01549_gb300", "csrc")
    for f in SWEEP_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_tag: str):
    """DRAM bytes per launch of the kernel from the committed ncu summary, or
    None if the kernel sources changed since it was captured."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tab = json.load(f)
    except Exception:
        return None
    ent = tab.get(kernel_tag)
    if not ent or ent.get("source_sha") != kernel_source_hash():
        return None
    return ent.get("bytes_per_launch")


def time_solves(S, b, variant, tol, maxit, steps, warmup):
    """Device time of `steps` solves (after `warmup`), from the library's events."""
    import torch
    from paper_1905_01549_gb300 import binding
    x = torch.zeros(S.n, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        x.zero_()
        S.solve(b, x0=x, variant=variant, tol=tol, maxit=maxit)
    torch.cuda.synchronize()
    dev_ms, iters, launches = [], [], 0
    res = None
    t0 = time.perf_counter()
    for _ in range(steps):
        x.zero_()
        res = S.solve(b, x0=x, variant=variant, tol=tol, maxit=maxit)
        dev_ms.append(res.init_ms + res.loop_ms)
        iters.append(res.iters)
        launches += binding.prcg_last_launches(S.handle)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return dict(dev_ms=dev_ms, iters=iters, launches=launches, wall=wall, last=res,
                loop_ms=res.loop_ms, status=res.status)


def aggregate_ranks(dev_s: float, iters: int, dist=None, device: str = "cuda"):
    """Whole-job numbers of a replica run: the slowest rank's time (max) and
    the iterations of all ranks (sum).  Single process: the inputs."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(dev_s), float(iters)
    import torch
    t = torch.tensor([float(dev_s)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    it = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    dist.all_reduce(it, op=dist.ReduceOp.SUM)
    return float(t.item()), float(it.item())


L2_BYTES = 129e6   # GB300 L2


def l2_note(n, nnz, bytes_it):
    """The timing rule this workload meets: inputs larger than L2 between
    timed iterations, or (small profiling cases) inputs that fit in it."""
    a = (12 * nnz + 4 * (n + 1)) / 1e9 if nnz else 0.0
    what = ("CSR %.2f GB + vectors" % a) if nnz else "matrix-free, vectors only"
    if bytes_it > L2_BYTES:
        return "inputs larger than L2 (%s; %.2f GB per iteration)" % (what, bytes_it / 1e9)
    return ("inputs fit in the 129 MB L2 (%s; %.1f MB per iteration): a cache-resident "
            "case, not an HBM measurement" % (what, bytes_it / 1e6))


def run_ours(args):
    import torch
    import paper_1905_01549_gb300 as G

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    prob = build_problem(args.workload)
    wl = f"{args.workload}_{args.op}_{args.precond}_{args.variant}"
    n = prob.n
    nnz = len(prob.csr[2]) if (prob.csr is not None and args.op == "csr") else 0
    op, precond, variant, tol = args.op, args.precond, args.variant, 1e-10
    maxit = 20000
    b_dev = torch.from_numpy(prob.b).cuda()
    S = make_solver(G, prob, op, precond)

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        main = time_solves(S, b_dev, variant, tol, maxit, args.steps, args.warmup)
    torch.cuda.synchronize()
    dev_s = sum(main["dev_ms"]) / 1e3
    tot_iters = sum(main["iters"])
    dev_s_max, all_iters = aggregate_ranks(dev_s, tot_iters, dist, "cuda")
    value = all_iters / dev_s_max
    K = main["iters"][-1]
    clocks = clk.summary()
    roof = sweep_roofline(S, variant, op, precond, n, nnz, sm_mhz=clocks.get("sm_mhz"))
    roof["traffic"] = ncu_traffic(f"{roof['kernel']}@{wl}")
    bytes_it = model_bytes(variant, op, precond, n, nnz)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "iters/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dev_s_max * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl, "n": n, "nnz": nnz, "operator": op, "precond": precond,
                   "variant": variant, "tol": tol, "iters_per_solve": K,
                   "step": "one complete solve to tol on resident inputs",
                   "l2": l2_note(n, nnz, bytes_it),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "iteration": {"us": main["loop_ms"] * 1e3 / max(K, 1),
                      "algorithmic_bytes": bytes_it,
                      "hbm_gbs": bytes_it / (main["loop_ms"] / 1e3 / max(K, 1)) / 1e9},
        "gpu_launches": main["launches"],
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extras:
        line["e2e"] = run_e2e(G, S, prob, variant, tol, maxit, args)
        line["variants"] = run_variants(G, prob, S, b_dev, args)
        line["batched"] = run_batched(G, args)
        line["mixed_precision"] = run_mixed(G, prob, args)
        line["autograd"] = run_autograd(G, args)
        line["convergence"] = run_convergence(G, args)
        line["dense_model"] = run_dense(G, args)
        line["sync_bound"] = run_sync_bound(G, args)
        if world == 1:
            line["cpu_baseline"] = run_cpu_baseline(prob, variant, precond, args)
    S.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e2e(G, S, prob, variant, tol, maxit, args):
    """Same metric through the C ABI with host (pinned) b and x: the
    host->device copy of b and x_0 and the device->host copy of x_K are
    inside each timed call."""
    import torch
    b_h = torch.from_numpy(prob.b).pin_memory()
    x_h = torch.zeros(prob.n, dtype=torch.float64).pin_memory()
    for _ in range(1):
        x_h.zero_()
        S.solve(b_h, x0=x_h, variant=variant, tol=tol, maxit=maxit)
    tot, iters = 0.0, 0
    for _ in range(max(2, args.steps // 2)):
        x_h.zero_()
        t0 = time.perf_counter()
        r = S.solve(b_h, x0=x_h, variant=variant, tol=tol, maxit=maxit)
        tot += time.perf_counter() - t0
        iters += r.iters
    return {"value": iters / tot, "unit": "iters/s", "h2d_bytes_per_step": 16 * prob.n,
            "d2h_bytes_per_step": 8 * prob.n + 256,
            "note": "prcg_solve with pinned host b, x; copies inside the timed call"}


def run_variants(G, prob, S_main, b_dev, args):
    """HS vs PR vs pipe-PR on the four cells of the 256^3 configuration (CSR
    and the matrix-free stencil, each with Jacobi and without a
    preconditioner), every solve to the same final relative residual 1e-10,
    and the 128^3 log-normal diffusion system."""
    peak, _ = _peaks()
    out = {}
    n = prob.n
    nnz = len(prob.csr[2])
    tol, maxit = 1e-10, 20000
    for op in ("csr", "stencil"):
        for precond in ("jacobi", "none"):
            main = op == "csr" and precond == args.precond and args.op == "csr"
            S = S_main if main else make_solver(G, prob, op, precond)
            cell = {}
            for variant in ("hs", "pr", "pipe_pr"):
                r = time_solves(S, b_dev, variant, tol, maxit, steps=2, warmup=1)
                K = r["iters"][-1]
                per = r["loop_ms"] / 1e3 / K
                by = model_bytes(variant, op, precond, n, nnz)
                rf = sweep_roofline(S, variant, op, precond, n, nnz if op == "csr" else 0)
                chk = S.solve(b_dev, variant=variant, tol=tol, maxit=maxit, history=True,
                              true_relres=True)
                cell[variant] = {
                    "iters_per_s": sum(r["iters"]) / (sum(r["dev_ms"]) / 1e3), "iters": K,
                    "final_relres": float(chk.hist[-1]), "final_true_relres": chk.true_relres,
                    "us_per_iter": per * 1e6, "algorithmic_gb_per_iter": by / 1e9,
                    "algorithmic_gbs": by / per / 1e9, "algorithmic_hbm_frac": by / per / 1e9 / peak,
                    "sweeps": rf["sweeps"], "status": r["status"], "jacobi_form": S.jacobi_form}
                out[f"{op}/{precond}/{variant}"] = cell[variant]
            out[f"{op}/{precond}/pr_over_hs"] = cell["pr"]["us_per_iter"] and \
                cell["hs"]["us_per_iter"] / cell["pr"]["us_per_iter"]
            if not main:
                S.close()
    # variable-coefficient diffusion 128^3, sigma = 2, Jacobi
    import torch
    vc = build_problem("varcoef3d_128")
    bvc = torch.from_numpy(vc.b).cuda()
    for op in ("csr", "varcoef"):
        S = make_solver(G, vc, "csr" if op == "csr" else "stencil", "jacobi")
        for variant in ("hs", "pr", "pipe_pr"):
            r = time_solves(S, bvc, variant, tol, maxit, steps=2, warmup=1)
            K = r["iters"][-1]
            per = r["loop_ms"] / 1e3 / K
            by = model_bytes(variant, op, "jacobi", vc.n, len(vc.csr[2]))
            out[f"varcoef128_{op}/jacobi/{variant}"] = {
                "iters_per_s": sum(r["iters"]) / (sum(r["dev_ms"]) / 1e3), "iters": K,
                "us_per_iter": per * 1e6, "achieved_gbs": by / per / 1e9,
                "frac_l2_note": "2M unknowns: vectors are 16.8 MB, partly L2-resident",
                "status": r["status"]}
        S.close()
    return out


def run_batched(G, args, count=512, config=None, plain=True):
    """`count` (512) shifted 2D Poisson systems (sides ~U{32..448}, shift
    ~U[0, 0.1], b ~ U(-1, 1)) in one persistent launch to 1e-8; autotuned
    configuration unless `config` = (cluster, threads) is given.  With
    `plain`, also the same systems one after another through prcg_solve."""
    import torch
    import problems as P
    spec = P.batch_spec(count)
    systems = [spec.system(i) for i in range(count)]
    nx = [s.dims[0] for s in systems]
    ny = [s.dims[1] for s in systems]
    B = G.BatchedSolver(nx, ny, spec.shifts)
    b = torch.from_numpy(np.concatenate([s.b for s in systems])).cuda()
    tol = 1e-8
    if config:
        cluster, threads = config
        B.configure(cluster, threads)
        table = []
    else:
        cluster, threads, _, table = B.tune(b, tol=tol)
    nbig, cluster_rest, threads_rest, clusters_rest = B.split()
    split = ({"nbig": nbig, "cluster_rest": cluster_rest, "threads_rest": threads_rest,
              "clusters_rest": clusters_rest} if nbig else None)
    ms = []
    for _ in range(max(2, args.steps)):
        x, iters, status, trr, worst, t = B.solve(b, tol=tol, true_relres=True)
        ms.append(t)
    B.close()
    best = min(ms)
    # FP64 issue floor: every row-iteration of the batched PR-CG kernel issues
    # 8 FP64 instructions without a preconditioner (sweep A: x, r, p and
    # <r, r>, which is also nu; sweep B: the FMA c p_i - sum of the 5-point
    # row, whose neighbour sum runs on the integer pipes, and three inner
    # products)
    sizes = np.array([x_ * y_ for x_, y_ in zip(nx, ny)], dtype=np.float64)
    row_iters = float((sizes * iters).sum())
    fp64 = 8.0 * row_iters
    out = {"solves_per_s": count / (best / 1e3), "ms": best, "cluster": cluster,
           "threads": threads, "split": split, "systems": count,
           "unknowns": int(sum(x_ * y_ for x_, y_ in zip(nx, ny))),
           "iters_total": int(iters.sum()), "iters_max": int(iters.max()),
           "all_converged": bool(np.all(status == 0)), "max_true_relres": float(trr.max()),
           "row_iterations": row_iters,
           "fp64_frac": fp64 / (best / 1e3) / fp64_peak(),
           "fp64_model": "8 FP64 instructions per row-iteration (the 5-point neighbour sum "
                         "runs on the integer pipes), peak 2 per SM per clock",
           "tuning": table}
    if not plain:
        return out
    # plain path: the same systems, one prcg_solve each (every 4th system, scaled)
    sel = list(range(0, count, 4))
    plain_ms = 0.0
    plain_iters = 0
    for i in sel:
        s = systems[i]
        with G.Solver.from_stencil(s.dims, diag_shift=s.shift) as S:
            bi = torch.from_numpy(s.b).cuda()
            S.solve(bi, tol=tol, maxit=100000)
            r = S.solve(bi, tol=tol, maxit=100000)
            plain_ms += r.init_ms + r.loop_ms
            plain_iters += r.iters
    plain_rate = len(sel) / (plain_ms / 1e3)
    out["plain_fp64_path"] = {"solves_per_s": plain_rate,
                              "sample": "every 4th system solved alone with prcg_solve "
                                        "(device time of init + loop), rate over the sample"}
    return out


def run_mixed(G, prob, args):
    """FP32-inner / FP64-refinement vs plain FP64 PR-CG, both to a true
    relative residual of 1e-8: 256^3 Poisson (stencil, Jacobi) and the
    Strakos diagonal (n = 1e5, lambda in [1e-3, 1e3], rho = 0.8)."""
    import torch
    import problems as P
    out = {}
    b = torch.from_numpy(prob.b).cuda()
    with G.Solver.from_stencil(prob.dims, precond="jacobi") as S:
        S.solve_refined_fp32(b, tol=1e-8)
        x, status, outer, inner, trr, hist, ms = S.solve_refined_fp32(b, tol=1e-8)
        S.solve(b, variant="pr", tol=1e-8, maxit=20000)
        r = S.solve(b, variant="pr", tol=1e-8, maxit=20000, true_relres=True)
        err = float((x - r.x).norm() / r.x.norm())
        out["poisson3d_256_stencil_jacobi"] = {
            "mixed_ms": ms, "outer": outer, "inner_iters": inner, "true_relres": trr,
            "fp64_ms": r.init_ms + r.loop_ms, "fp64_iters": r.iters, "fp64_true_relres": r.true_relres,
            "speedup": (r.init_ms + r.loop_ms) / ms, "rel_diff_vs_fp64_solution": err,
            "status": status}
    lam, bs = P.strakos_diagonal(100000, 1e-3, 1e3, 0.8)
    n = len(lam)
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    bb = torch.from_numpy(bs).cuda()
    xs = 1 / np.sqrt(n)
    with G.Solver.from_csr(rp, ci, lam) as S:
        S.solve_refined_fp32(bb, tol=1e-8)
        x, status, outer, inner, trr, hist, ms = S.solve_refined_fp32(bb, tol=1e-8)
        S.solve(bb, variant="pr", tol=1e-8, maxit=200000)
        r = S.solve(bb, variant="pr", tol=1e-8, maxit=200000, true_relres=True)
        out["strakos_diag_1e5"] = {
            "mixed_ms": ms, "outer": outer, "inner_iters": inner, "true_relres": trr,
            "err_vs_exact": float((x.cpu().numpy() - xs).__abs__().max() / xs),
            "fp64_ms": r.init_ms + r.loop_ms, "fp64_iters": r.iters,
            "fp64_err_vs_exact": float((r.x.cpu().numpy() - xs).__abs__().max() / xs),
            "speedup": (r.init_ms + r.loop_ms) / ms, "status": status}
    return out


def run_autograd(G, args):
    """Differentiation workload: 2D log-normal diffusion 512^2 (sigma = 2),
    loss = ||x - x_t||^2, gradients w.r.t. b and every face coefficient via
    the adjoint PR-CG solve (forward + backward to 1e-10, Jacobi)."""
    import torch
    import problems as P
    from paper_1905_01549_gb300.autograd import DiffusionSolver
    prob = P.varcoef2d(512, rhs="uniform", with_csr=False)
    xt = torch.tensor(P.rng_for("grad512_xt").standard_normal(prob.n), device="cuda")
    D = DiffusionSolver(prob.dims, precond="jacobi")
    ff = torch.tensor(prob.face_array(), device="cuda")
    bb = torch.tensor(prob.b, device="cuda")
    times = []
    for rep in range(3):
        fc = ff.clone().requires_grad_(True)
        bc = bb.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = D(fc, bc, tol=1e-10)
        ((x - xt) ** 2).sum().backward()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    res = D.solver.solve(bb, variant="pr", tol=1e-10, maxit=10 ** 6)
    D.close()
    return {"workload": "varcoef2d_512 sigma=2, loss=||x-x_t||^2, d/db and d/dfaces",
            "fwd_bwd_ms": min(times) * 1e3, "forward_iters": res.iters,
            "faces": int(ff.numel()), "grad_norm_faces": float(fc.grad.norm()),
            "grad_norm_b": float(bc.grad.norm())}


def paper_table2_model_48_8_3():
    """Table 2, row model_48_8_3, as printed in the paper (iterations to a
    10^5 A-norm error reduction, min log10 error), read from the fixture
    tests/golden/table2_model_48_8_3.txt; the paper's eigenvector draw is not
    known, so these are context, not expected values."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from golden import table2
    return table2()


def run_convergence(G, args):
    """Section 4's convergence study on the GPU variants: the Eq. 4.1 model
    problem (n = 48, rho = 0.8, kappa = 1e3, dense, passed as CSR), A-norm
    error of every iterate to k = 200, Table 2's two statistics."""
    import torch
    import problems as P
    from paper_1905_01549_gb300 import convergence
    prob = P.model_problem(48, 0.8, 1e3)
    n = prob.A.shape[0]
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    b = torch.from_numpy(prob.b).cuda()
    xs = torch.from_numpy(prob.x_star).cuda()
    out = {"workload": "model_48_8_3 (Eq. 4.1, Haar eigenvectors from the seeded generator), k <= 200"}
    t0 = time.perf_counter()
    paper = paper_table2_model_48_8_3()
    for pc in ("none", "jacobi"):
        with G.Solver.from_csr(rp, ci, np.ascontiguousarray(prob.A.ravel()), precond=pc) as S:
            st = convergence.study(S, b, xs, ["hs", "cgcg", "m", "pr", "gv", "pipe_m", "pipe_pr"], 200)
        out[pc] = {v: {"iters_to_1e5": r["iters_to_reduction"],
                       "min_log10_err": round(r["min_log10_err"], 2),
                       "paper": paper[pc][v]} for v, r in st.items()}
    out["seconds"] = round(time.perf_counter() - t0, 2)
    return out


def run_sync_bound(G, args):
    """The synchronisation-bound regime: 2D 5-point Poisson 64 x 64 (n = 4096),
    CSR, no preconditioner, x_true ~ U(-1, 1), b = A x_true, every variant to
    1e-10 (maxit 2n), as one persistent kernel and as the graph of sweeps.
    Device time of the whole solve (best of 5) and per iteration: the order
    follows the synchronisations per iteration (Table 1)."""
    import torch
    import problems as P
    prob = P.poisson2d_64()
    rp, ci, v = prob.csr
    b = torch.from_numpy(prob.b).cuda()
    out = {"workload": "poisson2d_64 CSR, no preconditioner, tol 1e-10, maxit 2n"}
    saved = os.environ.get("PRCG_PERSIST_MAX")
    try:
        for path, bound in (("persistent", str(1 << 21)), ("graph", "0")):
            os.environ["PRCG_PERSIST_MAX"] = bound
            row = {}
            with G.Solver.from_csr(rp, ci, v) as S:
                for var in ("hs", "cgcg", "m", "pr", "gv", "pipe_m", "pipe_pr"):
                    best = None
                    for _ in range(5):
                        r = S.solve(b, variant=var, tol=1e-10, maxit=2 * prob.n)
                        t = r.init_ms + r.loop_ms
                        if best is None or t < best[0]:
                            best = (t, r.iters, r.status)
                    row[var] = {"ms": round(best[0], 4), "iters": best[1], "status": best[2],
                                "us_per_iter": round(1e3 * best[0] / max(best[1], 1), 2)}
            out[path] = row
    finally:
        if saved is None:
            os.environ.pop("PRCG_PERSIST_MAX", None)
        else:
            os.environ["PRCG_PERSIST_MAX"] = saved
    return out


def run_dense(G, args):
    """Section 5's workload on one GPU: the Eq. 4.1 model problem with
    n = 10752, rho = 0.9, kappa = 1e6 stored as a dense matrix, no
    preconditioner, 1000 iterations of each variant with only the main loop
    timed (minimum over 3 runs), as the paper times it.  Per iteration the
    product reads A once (n^2 x 8 B); pipe-PR-CG and pipe-M-CG form the
    paired product [A s, A r] in that one pass, at twice the FP64 FMAs."""
    import torch
    import problems as P
    n, iters = 10752, 1000
    t0 = time.perf_counter()
    A, b, _ = P.model_problem_on_device(n, 0.9, 1e6)
    gen_s = time.perf_counter() - t0
    S = G.Solver.from_dense(A)
    del A
    torch.cuda.empty_cache()
    peak_hbm, _ = _peaks()
    peak_fp = fp64_peak()
    out = {"workload": "model problem Eq. 4.1, n=10752, rho=0.9, kappa=1e6, dense FP64, no precond",
           "iterations": iters, "generation_s": round(gen_s, 1)}
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    for v in ("hs", "cgcg", "m", "pr", "gv", "pipe_m", "pipe_pr"):
        best = None
        for _ in range(3):
            x.zero_()
            res = S.solve(b, x0=x, variant=v, tol=0.0, maxit=iters)
            if best is None or res.loop_ms < best.loop_ms:
                best = res
        k = max(best.iters, 1)
        us = 1e3 * best.loop_ms / k
        products = 2 if v in ("pipe_pr", "pipe_m") else 1
        fma = products * float(n) * n
        out[v] = {"us_per_iter": round(us, 2), "iters": best.iters, "status": best.status,
                  "A_read_gbs": round(8.0 * n * n / (us * 1e-6) / 1e9, 1),
                  "hbm_frac": round(8.0 * n * n / (us * 1e-6) / 1e9 / peak_hbm, 3),
                  "fp64_frac": round(fma / (us * 1e-6) / peak_fp, 3)}
    S.close()
    return out


def host_cores() -> int:
    """Host cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def c_oracle_loop(prob, variant, precond, iters, threads):
    """Seconds of the main loop (initialize() excluded) of `iters` iterations
    of the multi-threaded C oracle (oracle/cg_oracle.c), and its K."""
    import scipy.sparse as sp
    import oracle as O
    from oracle import c_oracle as C
    d = None
    if precond == "jacobi":
        rp, ci, v = prob.csr
        d = O.jacobi_inverse_diagonal(sp.csr_matrix((v, ci, rp), shape=(prob.n, prob.n)))
    res = C.solve(variant, prob.csr, prob.b, d=d, tol=0.0, maxit=iters, threads=threads)
    return res.loop_s, res.iters


def cpu_sample_plan(prob, variant, precond, threads, budget_s=15.0, trials=3):
    """Iterations per trial so that `trials` trials take about budget_s."""
    t, k = c_oracle_loop(prob, variant, precond, 3, threads)
    per = t / max(k, 1)
    return int(min(200, max(5, budget_s / trials / max(per, 1e-6))))


def run_cpu_baseline(prob, variant, precond, args):
    """The C oracle on every host core: main loop only (initialize() timed
    separately inside the oracle and left out, as the paper times only the
    main loop), the minimum over 3 trials."""
    cores = host_cores()
    iters = cpu_sample_plan(prob, variant, precond, cores)
    best = None
    for _ in range(3):
        t, k = c_oracle_loop(prob, variant, precond, iters, cores)
        best = t if best is None else min(best, t)
    return {"value": iters / best, "unit": "iters/s", "cores": cores, "kind": "oracle",
            "sample": f"{iters} {variant.upper()}-CG iterations of the same {args.workload} "
                      f"{args.op} {precond} system, C oracle (OpenMP, {cores} threads = the "
                      f"process's CPU affinity, plain FP64 loops, CSR matvec); main loop only, "
                      f"minimum of 3 trials ({best:.2f} s)"}


def run_reference(args):
    """The oracle as the reference arm: the multi-threaded C oracle on every
    host core, each step a bounded sample (the main loop of a fixed number of
    iterations; initialize() is excluded and timed apart) of the same
    workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = build_problem(args.workload)
    variant, precond = args.variant, args.precond
    cores = host_cores()
    per = cpu_sample_plan(prob, variant, precond, cores, budget_s=8.0, trials=1)
    for _ in range(args.warmup):
        c_oracle_loop(prob, variant, precond, 1, cores)
    tot, its = 0.0, 0
    for _ in range(args.steps):
        t, k = c_oracle_loop(prob, variant, precond, per, cores)
        tot += t
        its += k
    value = its / tot
    stands_in = "; the CSR operator stands in for the stencil" if args.op == "stencil" else ""
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{args.workload}_{args.op}_{precond}_{variant}", "n": prob.n,
                       "nnz": len(prob.csr[2]), "operator": "csr", "precond": precond,
                       "variant": variant, "tol": 1e-10},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: the main loop of {per} {variant.upper()}-CG "
                                       f"iterations of the C oracle (OpenMP, {cores} threads; "
                                       f"initialize() excluded){stands_in}"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="poisson3d_256",
                    help="problem: poisson3d_256, poisson3d_<N>, varcoef3d_128")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--op", default="csr", choices=["csr", "stencil"])
    ap.add_argument("--variant", default="pr", choices=["pr", "hs", "pipe_pr", "m", "pipe_m"])
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "none"])
    ap.add_argument("--batched-only", type=int, default=0, metavar="COUNT",
                    help="time only the batched solver on COUNT systems (a profiling case)")
    ap.add_argument("--batched-config", default="", metavar="CLUSTER,THREADS",
                    help="with --batched-only: this launch configuration instead of the tuner")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import __graft_entry__
    __graft_entry__.build()
    if args.batched_only:
        import paper_1905_01549_gb300 as G
        cfg = tuple(int(v) for v in args.batched_config.split(",")) if args.batched_config else None
        res = run_batched(G, args, count=args.batched_only, config=cfg, plain=False)
        print(json.dumps({"batched": res}), flush=True)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
