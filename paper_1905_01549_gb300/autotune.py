"""Autotuner for the batched persistent solver's launch configuration.

The batched kernel (csrc/prcg_batched.cu) runs one PR-CG solver per
thread-block cluster; the best cluster size (1..16 CTAs) and CTA size
depend on the size mix of the batch: small systems want many independent
solvers, large ones want several SMs per system so the largest solve does
not set the makespan.  A split launch serves both: the costliest systems on
large clusters beside the rest on smaller ones.  The tuner times each candidate on the batch itself
(the device time of the solve's graph launch, CUDA events), keeps the
fastest and caches the choice in a JSON file keyed by the batch's shape.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Iterable, Optional, Sequence, Tuple

from . import binding

DEFAULT_CANDIDATES: Tuple[Tuple[int, int], ...] = (
    (1, 256), (1, 512), (1, 1024), (2, 256), (2, 512), (4, 256), (4, 512), (8, 256), (8, 512),
    (8, 1024), (16, 256), (16, 512), (16, 1024))

# Split launches (nbig, cluster_big, threads_big, cluster_rest, threads_rest):
# the nbig costliest systems on 16-CTA clusters beside the rest on 8-CTA
# clusters, for batches whose largest systems set the makespan.
DEFAULT_SPLITS: Tuple[Tuple[int, int, int, int, int], ...] = (
    (2, 16, 512, 8, 512), (4, 16, 512, 8, 512), (8, 16, 512, 8, 512), (16, 16, 512, 8, 512))


def default_cache_path() -> str:
    base = os.environ.get("PRCG_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "prcg_gb300", "batched_tuning.json")


_KERNEL_SOURCES = ("prcg_batched.cu", "prcg_reduce.cuh")


def kernel_tag() -> str:
    """Fingerprint of the batched kernel's sources: a cached choice is only
    reused for the kernel it was measured on."""
    h = hashlib.sha256()
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    for f in _KERNEL_SOURCES:
        try:
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
        except OSError:
            h.update(f.encode())
    return h.hexdigest()[:12]


def batch_key(nx: Sequence[int], ny: Sequence[int], shift: Sequence[float], precond: int,
              tol: float, device: str = "") -> str:
    """Cache key: the batch's shape, preconditioner and tolerance, the kernel
    version and the device the choice was measured on."""
    h = hashlib.sha256()
    for arr in (nx, ny):
        h.update(",".join(str(int(v)) for v in arr).encode())
    h.update(",".join(f"{float(v):.6g}" for v in shift).encode())
    h.update(f"{precond}:{tol:.3g}:{device}:{kernel_tag()}".encode())
    return h.hexdigest()[:24]


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _apply(bt, cluster, threads, split):
    if split:
        nbig, cluster_rest, threads_rest = split
        binding.prcg_batched_configure_split(bt, nbig, cluster, threads, cluster_rest, threads_rest)
    else:
        binding.prcg_batched_configure(bt, cluster, threads)


def tune(bt, b, x0, tol: float, maxit: int, key: Optional[str] = None,
         candidates: Iterable[Tuple[int, int]] = DEFAULT_CANDIDATES,
         splits: Iterable[Tuple[int, int, int, int, int]] = DEFAULT_SPLITS, reps: int = 1,
         cache_path: Optional[str] = None, use_cache: bool = True):
    """Pick the launch configuration of batch handle `bt`: one launch of
    (cluster, threads) from `candidates`, or a split launch from `splits`.
    Returns (cluster, threads, ms, table); for a split winner cluster and
    threads are those of its first launch (prcg_batched_split gives the
    rest).  Table rows: (cluster, threads, ms) and (nbig, cluster_big,
    threads_big, cluster_rest, threads_rest, ms); ms is None where the
    configuration could not be launched.

    b and x0 are the batch's concatenated right-hand side and initial guess
    (x0 is copied for every trial and left unchanged)."""
    import torch
    cache_path = cache_path or default_cache_path()
    cache = _load(cache_path) if use_cache else {}
    if key and use_cache and key in cache:
        ent = cache[key]
        _apply(bt, ent["cluster"], ent["threads"], ent.get("split"))
        return ent["cluster"], ent["threads"], ent["ms"], ent.get("table", [])
    table = []
    best = None   # (cluster, threads, split or None, ms)
    x = torch.empty_like(x0)

    def trial():
        times = []
        for _ in range(reps + 1):   # first run instantiates the graph
            x.copy_(x0)
            binding.prcg_batched_solve(bt, b, x, tol, maxit)
            times.append(binding.prcg_batched_last_ms(bt))
        return min(times[1:]) if reps > 0 else times[0]

    for cluster, threads in candidates:
        try:
            binding.prcg_batched_configure(bt, cluster, threads)
        except binding.PrcgError:
            table.append((cluster, threads, None))
            continue
        ms = trial()
        table.append((cluster, threads, ms))
        if best is None or ms < best[3]:
            best = (cluster, threads, None, ms)
    for nbig, cb, tb, cr, tr in splits:
        try:
            binding.prcg_batched_configure_split(bt, nbig, cb, tb, cr, tr)
        except binding.PrcgError:
            table.append((nbig, cb, tb, cr, tr, None))
            continue
        ms = trial()
        table.append((nbig, cb, tb, cr, tr, ms))
        if best is None or ms < best[3]:
            best = (cb, tb, (nbig, cr, tr), ms)
    if best is None:
        raise RuntimeError("no batched configuration could be launched")
    _apply(bt, best[0], best[1], best[2])
    if key:
        cache = _load(cache_path)
        cache[key] = {"cluster": best[0], "threads": best[1], "ms": best[3], "table": table,
                      "split": list(best[2]) if best[2] else None}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return best[0], best[1], best[3], table
