"""ctypes wrapper of the multi-threaded C oracle (oracle/cg_oracle.c).

TEST INFRASTRUCTURE ONLY: loaded by the tests and by the CPU legs of
bench.py.  ``build()`` compiles the shared library with gcc and OpenMP
(plain FP64, no contraction); ``solve()`` runs HS-CG (Algorithm 1), PR-CG
(Algorithm 2) or pipe-PR-CG (Algorithm 3) on a CSR matrix.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cg_oracle.c")
LIB = os.path.join(HERE, "libcg_oracle.so")
VARIANT_IDS = {"hs": 0, "pr": 1, "pipe_pr": 2}

_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=199309L", "-fopenmp",
           "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("gcc failed for the C oracle:\n" + res.stderr)
    os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(LIB)
        vp = ctypes.c_void_p
        lib.cgo_solve.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), vp,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.cgo_solve.restype = ctypes.c_int
        lib.cgo_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclasses.dataclass
class CResult:
    x: np.ndarray
    iters: int
    status: int
    hist: Optional[np.ndarray]
    init_s: float
    loop_s: float


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def solve(variant: str, csr, b, d=None, x0=None, tol: float = 0.0, maxit: int = 100,
          threads: int = 0, history: bool = False) -> CResult:
    """csr = (row_ptr int32, col_idx int32, vals float64); d = Jacobi vector or None."""
    rp, ci, va = (np.ascontiguousarray(csr[0], dtype=np.int32),
                  np.ascontiguousarray(csr[1], dtype=np.int32),
                  np.ascontiguousarray(csr[2], dtype=np.float64))
    n = len(rp) - 1
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    dd = None if d is None else np.ascontiguousarray(d, dtype=np.float64)
    hist = np.full(maxit + 1, np.nan) if history else None
    k = ctypes.c_int(0)
    ti, tl = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = load().cgo_solve(VARIANT_IDS[variant], n, _p(rp), _p(ci), _p(va), _p(dd), _p(b), _p(x),
                          float(tol), int(maxit), int(threads), ctypes.byref(k), _p(hist),
                          ctypes.byref(ti), ctypes.byref(tl))
    if st < 0:
        raise ValueError("cgo_solve rejected its arguments")
    return CResult(x, k.value, st, None if hist is None else hist[:k.value + 1], ti.value, tl.value)


def max_threads() -> int:
    return load().cgo_max_threads()
