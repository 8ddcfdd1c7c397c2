"""ctypes binding of libprcg.so: the C ABI of include/prcg.h, same names.

Argument marshalling only: arrays are passed as raw pointers (torch tensors
on the GPU or the host, or numpy arrays), every computation happens in the
CUDA library.  There is no CPU fallback: if the library is missing the
import of this module fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libprcg.so")

(PRCG_HS, PRCG_PR, PRCG_PIPE_PR, PRCG_M, PRCG_PIPE_M, PRCG_CGCG, PRCG_GV,
 PRCG_PR_NO_RECOMPUTE, PRCG_PIPE_PR_NO_RECOMPUTE) = range(9)
PRCG_PRECOND_NONE, PRCG_PRECOND_JACOBI = 0, 1
PRCG_OK, PRCG_NOT_CONVERGED, PRCG_BREAKDOWN = 0, 1, 2
PRCG_ERR_INVALID, PRCG_ERR_CUDA, PRCG_ERR_OOM, PRCG_ERR_TIMEOUT, PRCG_ERR_UNSUPPORTED = \
    -1, -2, -3, -4, -5

VARIANT_IDS = {"hs": PRCG_HS, "pr": PRCG_PR, "pipe_pr": PRCG_PIPE_PR, "m": PRCG_M,
               "pipe_m": PRCG_PIPE_M, "cgcg": PRCG_CGCG, "gv": PRCG_GV,
               # the no-recompute ablations of Section 3 (Figs. 1 and 2)
               "pr_norecompute": PRCG_PR_NO_RECOMPUTE,
               "pipe_pr_norecompute": PRCG_PIPE_PR_NO_RECOMPUTE}
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", 2: "BREAKDOWN", -1: "ERR_INVALID", -2: "ERR_CUDA",
                -3: "ERR_OOM", -4: "ERR_TIMEOUT", -5: "ERR_UNSUPPORTED"}

# every symbol include/prcg.h declares
EXPORTS = ("prcg_create_csr", "prcg_create_stencil", "prcg_create_dense", "prcg_solve", "prcg_last_timing",
           "prcg_time_sweeps", "prcg_solve_f32_refined", "prcg_update_faces",
           "prcg_grad_faces", "prcg_grad_csr_values",
           "prcg_last_launches", "prcg_destroy", "prcg_last_error", "prcg_n", "prcg_error_anorm",
           "prcg_jacobi_form", "prcg_int_diagonal", "prcg_last_fixed_sweeps",
           "prcg_trace_enable", "prcg_trace_get", "prcg_check_guards",
           "prcg_inject_barrier_skip", "prcg_test_neighbour_sum",
           "prcg_pr_solve_stencil_noalloc", "prcg_batched_create", "prcg_batched_configure",
           "prcg_batched_configure_split", "prcg_batched_split",
           "prcg_batched_solve", "prcg_batched_last_ms", "prcg_batched_config",
           "prcg_batched_last_error", "prcg_batched_destroy")


class PrcgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_float_p = ctypes.POINTER(ctypes.c_float)

_lib: Optional[ctypes.CDLL] = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libprcg.so and declare the signatures; raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1905_01549_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.prcg_create_csr.argtypes = [ctypes.POINTER(vp), ctypes.c_int64, ctypes.c_int64, vp, vp, vp,
                                    ctypes.c_int, vp]
    lib.prcg_create_csr.restype = ctypes.c_int
    lib.prcg_create_stencil.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_double,
                                        ctypes.c_int, vp]
    lib.prcg_create_stencil.restype = ctypes.c_int
    lib.prcg_create_dense.argtypes = [ctypes.POINTER(vp), ctypes.c_int64, vp, ctypes.c_int, vp]
    lib.prcg_create_dense.restype = ctypes.c_int
    lib.prcg_solve.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_double, ctypes.c_int, vp,
                               _c_int_p, _c_double_p]
    lib.prcg_solve.restype = ctypes.c_int
    lib.prcg_last_timing.argtypes = [vp, _c_float_p, _c_float_p, _c_int_p]
    lib.prcg_last_timing.restype = ctypes.c_int
    lib.prcg_solve_f32_refined.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_int, _c_int_p, _c_int_p,
                                           _c_double_p, vp]
    lib.prcg_solve_f32_refined.restype = ctypes.c_int
    lib.prcg_update_faces.argtypes = [vp, vp, ctypes.c_double]
    lib.prcg_update_faces.restype = ctypes.c_int
    lib.prcg_grad_faces.argtypes = [vp, vp, vp, vp]
    lib.prcg_grad_faces.restype = ctypes.c_int
    lib.prcg_grad_csr_values.argtypes = [vp, vp, vp, vp]
    lib.prcg_grad_csr_values.restype = ctypes.c_int
    lib.prcg_time_sweeps.argtypes = [vp, ctypes.c_int, ctypes.c_int, _c_float_p, _c_int_p]
    lib.prcg_time_sweeps.restype = ctypes.c_int
    lib.prcg_last_launches.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.prcg_last_launches.restype = ctypes.c_int
    lib.prcg_destroy.argtypes = [vp]
    lib.prcg_destroy.restype = ctypes.c_int
    lib.prcg_last_error.argtypes = [vp]
    lib.prcg_last_error.restype = ctypes.c_char_p
    lib.prcg_n.argtypes = [vp]
    lib.prcg_n.restype = ctypes.c_int64
    lib.prcg_jacobi_form.argtypes = [vp]
    lib.prcg_jacobi_form.restype = ctypes.c_int
    lib.prcg_int_diagonal.argtypes = [vp]
    lib.prcg_int_diagonal.restype = ctypes.c_int
    lib.prcg_last_fixed_sweeps.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.prcg_last_fixed_sweeps.restype = ctypes.c_int
    lib.prcg_error_anorm.argtypes = [vp, vp, vp, _c_double_p]
    lib.prcg_error_anorm.restype = ctypes.c_int
    lib.prcg_inject_barrier_skip.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64]
    lib.prcg_inject_barrier_skip.restype = ctypes.c_int
    lib.prcg_check_guards.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.prcg_test_neighbour_sum.argtypes = [ctypes.c_int, vp, ctypes.c_int64, vp]
    lib.prcg_test_neighbour_sum.restype = ctypes.c_int
    lib.prcg_check_guards.restype = ctypes.c_int
    lib.prcg_trace_enable.argtypes = [vp, ctypes.c_int]
    lib.prcg_trace_enable.restype = ctypes.c_int
    lib.prcg_trace_get.argtypes = [vp, vp, ctypes.c_int]
    lib.prcg_trace_get.restype = ctypes.c_int
    lib.prcg_pr_solve_stencil_noalloc.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                                  ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                                  vp, vp, ctypes.c_double, ctypes.c_int, vp,
                                                  _c_int_p, vp]
    lib.prcg_pr_solve_stencil_noalloc.restype = ctypes.c_int
    lib.prcg_batched_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, vp, vp, ctypes.c_int, vp]
    lib.prcg_batched_create.restype = ctypes.c_int
    lib.prcg_batched_configure.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.prcg_batched_configure.restype = ctypes.c_int
    lib.prcg_batched_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int, vp, vp, vp]
    lib.prcg_batched_solve.restype = ctypes.c_int
    lib.prcg_batched_last_ms.argtypes = [vp, _c_float_p]
    lib.prcg_batched_last_ms.restype = ctypes.c_int
    lib.prcg_batched_config.argtypes = [vp, _c_int_p, _c_int_p, _c_int_p]
    lib.prcg_batched_config.restype = ctypes.c_int
    lib.prcg_batched_configure_split.argtypes = [vp] + [ctypes.c_int] * 5
    lib.prcg_batched_configure_split.restype = ctypes.c_int
    lib.prcg_batched_split.argtypes = [vp, _c_int_p, _c_int_p, _c_int_p, _c_int_p]
    lib.prcg_batched_split.restype = ctypes.c_int
    lib.prcg_batched_last_error.argtypes = [vp]
    lib.prcg_batched_last_error.restype = ctypes.c_char_p
    lib.prcg_batched_destroy.argtypes = [vp]
    lib.prcg_batched_destroy.restype = ctypes.c_int
    _lib = lib
    return lib


def ptr(a) -> Optional[int]:
    """Raw address of a torch tensor / numpy array (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("array must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(code: int, ctx=None):
    if code < 0:
        msg = load().prcg_last_error(ctx).decode(errors="replace")
        raise PrcgError(code, msg)
    return code


def prcg_create_csr(n, nnz, row_ptr, col_idx, vals, precond=PRCG_PRECOND_NONE, stream=None):
    """Create a CSR context; returns the opaque handle (an int)."""
    lib = load()
    out = ctypes.c_void_p()
    rc = lib.prcg_create_csr(ctypes.byref(out), int(n), int(nnz), ptr(row_ptr), ptr(col_idx),
                             ptr(vals), int(precond), _stream_ptr(stream))
    _check(rc, None)
    return out.value


def prcg_create_stencil(dim, nx, ny, nz, face_coeff=None, diag_shift=0.0,
                        precond=PRCG_PRECOND_NONE, stream=None):
    """Create a matrix-free stencil context; returns the opaque handle."""
    lib = load()
    out = ctypes.c_void_p()
    rc = lib.prcg_create_stencil(ctypes.byref(out), int(dim), int(nx), int(ny), int(nz),
                                 ptr(face_coeff), float(diag_shift), int(precond),
                                 _stream_ptr(stream))
    _check(rc, None)
    return out.value


def prcg_create_dense(n, A, precond=PRCG_PRECOND_NONE, stream=None):
    """Create a dense symmetric matrix context (A: n x n, row-major, host or
    device); returns the opaque handle."""
    lib = load()
    out = ctypes.c_void_p()
    rc = lib.prcg_create_dense(ctypes.byref(out), int(n), ptr(A), int(precond), _stream_ptr(stream))
    _check(rc, None)
    return out.value


def prcg_solve(ctx, variant, b, x, tol, maxit, residual_history=None, want_true_relres=False):
    """Solve in place (x: in x_0, out x_K); returns (status, iters, true_relres or None)."""
    lib = load()
    iters = ctypes.c_int(0)
    trr = ctypes.c_double(float("nan"))
    rc = lib.prcg_solve(ctx, int(variant), ptr(b), ptr(x), float(tol), int(maxit),
                        ptr(residual_history), ctypes.byref(iters),
                        ctypes.byref(trr) if want_true_relres else None)
    _check(rc, ctx)
    return rc, iters.value, (trr.value if want_true_relres else None)


def prcg_last_timing(ctx):
    """(init_ms, loop_ms, iters) of the last solve, from CUDA events."""
    lib = load()
    a, b, k = ctypes.c_float(), ctypes.c_float(), ctypes.c_int()
    _check(lib.prcg_last_timing(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(k)), ctx)
    return a.value, b.value, k.value


def prcg_solve_f32_refined(ctx, b, x, tol, max_outer, inner_tol, inner_maxit, outer_history=None):
    """FP32 inner / FP64 refinement solve; returns (status, outer, inner_total, true_relres)."""
    o, it, trr = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    rc = load().prcg_solve_f32_refined(ctx, ptr(b), ptr(x), float(tol), int(max_outer),
                                       float(inner_tol), int(inner_maxit), ctypes.byref(o),
                                       ctypes.byref(it), ctypes.byref(trr), ptr(outer_history))
    _check(rc, ctx)
    return rc, o.value, it.value, trr.value


def prcg_update_faces(ctx, face_coeff, diag_shift=0.0):
    return _check(load().prcg_update_faces(ctx, ptr(face_coeff), float(diag_shift)), ctx)


def prcg_grad_faces(ctx, lam, x, grad_faces):
    return _check(load().prcg_grad_faces(ctx, ptr(lam), ptr(x), ptr(grad_faces)), ctx)


def prcg_grad_csr_values(ctx, lam, x, grad_vals):
    return _check(load().prcg_grad_csr_values(ctx, ptr(lam), ptr(x), ptr(grad_vals)), ctx)


def prcg_time_sweeps(ctx, variant, reps):
    """Average ms of each sweep of one iteration (list of 1 to 3 floats)."""
    buf = (ctypes.c_float * 3)()
    k = ctypes.c_int()
    _check(load().prcg_time_sweeps(ctx, int(variant), int(reps), buf, ctypes.byref(k)), ctx)
    return [buf[i] for i in range(k.value)]


def prcg_last_launches(ctx) -> int:
    """Kernels the last solve launched."""
    k = ctypes.c_int64()
    _check(load().prcg_last_launches(ctx, ctypes.byref(k)), ctx)
    return k.value


def prcg_destroy(ctx):
    return load().prcg_destroy(ctx)


def prcg_last_error(ctx=None) -> str:
    return load().prcg_last_error(ctx).decode(errors="replace")


def prcg_n(ctx) -> int:
    return int(load().prcg_n(ctx))


def prcg_inject_barrier_skip(ctx, cta: int, barrier: int, spin_limit: int = 1 << 16):
    """Test hook: in the next persistent solve, CTA `cta` skips grid barrier
    `barrier`, so the solve ends with PRCG_ERR_TIMEOUT (see prcg.h)."""
    _check(load().prcg_inject_barrier_skip(ctx, int(cta), int(barrier), int(spin_limit)), ctx)


def prcg_check_guards(ctx) -> int:
    """Number of corrupted guard words of the context (0 = no out-of-bounds write)."""
    bad = ctypes.c_int64(0)
    _check(load().prcg_check_guards(ctx, ctypes.byref(bad)), ctx)
    return int(bad.value)


def prcg_test_neighbour_sum(v) -> "np.ndarray":
    """The stencil's device neighbour sum of each row of v (float64, shape
    (count, 4) or (count, 6)); a test hook for that kernel arithmetic."""
    import numpy as np
    v = np.ascontiguousarray(v, dtype=np.float64)
    if v.ndim != 2:
        raise ValueError("v must be (count, terms)")
    out = np.empty(v.shape[0], dtype=np.float64)
    _check(load().prcg_test_neighbour_sum(int(v.shape[1]), v.ctypes.data, int(v.shape[0]),
                                          out.ctypes.data), None)
    return out


TRACE_FIELDS = ("alpha", "beta", "nu", "nu_pred", "mu", "sigma", "gamma", "rho", "eta", "unused")


def prcg_trace_enable(ctx, on: bool):
    _check(load().prcg_trace_enable(ctx, 1 if on else 0), ctx)


def prcg_trace_get(ctx, slots: int) -> np.ndarray:
    """The last solve's scalar trace as a (slots', 10) array (see prcg.h)."""
    out = np.empty((max(slots, 0), len(TRACE_FIELDS)))
    m = load().prcg_trace_get(ctx, ptr(out), int(slots))
    _check(m if m < 0 else 0, ctx)
    return out[:m]


def prcg_last_fixed_sweeps(ctx) -> int:
    """Product sweeps of the last solve that read the fixed-point copy of p."""
    v = ctypes.c_int64(0)
    _check(load().prcg_last_fixed_sweeps(ctx, ctypes.byref(v)), ctx)
    return v.value


def prcg_jacobi_form(ctx) -> int:
    """0 no preconditioner, 1 scalar d, 2 vector d."""
    rc = load().prcg_jacobi_form(ctx)
    _check(rc if rc < 0 else 0, ctx)
    return rc


def prcg_int_diagonal(ctx) -> int:
    """The constant stencil's integer diagonal used by the integer product rows, or 0."""
    rc = load().prcg_int_diagonal(ctx)
    _check(rc if rc < 0 else 0, ctx)
    return rc


def prcg_error_anorm(ctx, x_star, x) -> float:
    """||x* - x||_A with the context's operator (host or device arrays)."""
    err = ctypes.c_double(0.0)
    _check(load().prcg_error_anorm(ctx, ptr(x_star), ptr(x), ctypes.byref(err)), ctx)
    return err.value


def prcg_pr_solve_stencil_noalloc(dim, nx, ny, nz, diag_shift, precond, b, x, tol, maxit,
                                  residual_history=None, stream=None):
    """PR-CG without device allocation (n <= 65536, device b / x);
    returns (status, iters).  Raises PrcgError on a negative status."""
    iters = ctypes.c_int(0)
    rc = load().prcg_pr_solve_stencil_noalloc(int(dim), int(nx), int(ny), int(nz),
                                              float(diag_shift), int(precond), ptr(b), ptr(x),
                                              float(tol), int(maxit), ptr(residual_history),
                                              ctypes.byref(iters), _stream_ptr(stream))
    if rc < 0:
        raise PrcgError(rc, "prcg_pr_solve_stencil_noalloc failed")
    return rc, iters.value


def _bcheck(code, bt):
    if code < 0:
        msg = load().prcg_batched_last_error(bt).decode(errors="replace") if bt else ""
        raise PrcgError(code, msg or "batched call failed")
    return code


def prcg_batched_create(nx, ny, shift, precond=PRCG_PRECOND_NONE, stream=None):
    """Create a batch of shifted 2D 5-point systems; returns the handle."""
    nx = np.ascontiguousarray(nx, dtype=np.int32)
    ny = np.ascontiguousarray(ny, dtype=np.int32)
    shift = np.ascontiguousarray(shift, dtype=np.float64)
    out = ctypes.c_void_p()
    _bcheck(load().prcg_batched_create(ctypes.byref(out), len(nx), ptr(nx), ptr(ny), ptr(shift),
                                       int(precond), _stream_ptr(stream)), None)
    return out.value


def prcg_batched_configure(bt, cluster, threads):
    return _bcheck(load().prcg_batched_configure(bt, int(cluster), int(threads)), bt)


def prcg_batched_configure_split(bt, nbig, cluster_big, threads_big, cluster_rest, threads_rest):
    return _bcheck(load().prcg_batched_configure_split(bt, int(nbig), int(cluster_big),
                                                       int(threads_big), int(cluster_rest),
                                                       int(threads_rest)), bt)


def prcg_batched_split(bt):
    """(nbig, cluster_rest, threads_rest, clusters_rest); zeros for one launch."""
    v = [ctypes.c_int() for _ in range(4)]
    _bcheck(load().prcg_batched_split(bt, *[ctypes.byref(t) for t in v]), bt)
    return tuple(t.value for t in v)


def prcg_batched_solve(bt, b, x, tol, maxit, iters=None, status=None, true_relres=None):
    """Solve every system of the batch; returns the worst status."""
    return _bcheck(load().prcg_batched_solve(bt, ptr(b), ptr(x), float(tol), int(maxit), ptr(iters),
                                             ptr(status), ptr(true_relres)), bt)


def prcg_batched_last_ms(bt) -> float:
    ms = ctypes.c_float()
    _bcheck(load().prcg_batched_last_ms(bt, ctypes.byref(ms)), bt)
    return ms.value


def prcg_batched_config(bt):
    c, t, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcheck(load().prcg_batched_config(bt, ctypes.byref(c), ctypes.byref(t), ctypes.byref(k)), bt)
    return c.value, t.value, k.value


def prcg_batched_last_error(bt) -> str:
    return load().prcg_batched_last_error(bt).decode(errors="replace")


def prcg_batched_destroy(bt):
    return load().prcg_batched_destroy(bt)
