"""CPU oracle for the predict-and-recompute CG variants (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package; the CUDA library shares no code
with it.  See ``cg_variants`` for the algorithms and ``adjoint`` /
``refinement`` for the differentiation and mixed-precision forms.
"""
from .cg_variants import (OK, NOT_CONVERGED, BREAKDOWN, VARIANTS, SOLVERS, Result,  # noqa: F401
                          solve, hs_cg, pr_cg, pipe_pr_cg, m_cg, pipe_m_cg, cg_cg, gv_cg,
                          jacobi_inverse_diagonal, true_relres, a_norm_error, as_operator)
from .refinement import refined_fp32  # noqa: F401,E402
from . import adjoint  # noqa: F401,E402
