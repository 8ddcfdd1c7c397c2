/*
 * prcg.h -- C ABI of the GB300 (sm_103a) predict-and-recompute CG library.
 *
 * The library solves A x = b for a symmetric positive definite A, optionally
 * with a symmetric positive definite preconditioner M^{-1} (Section 1 of
 * Chen & Carson, "Predict-and-recompute conjugate gradient variants": the
 * methods need only products with A and M^{-1}).  The caller supplies A,
 * the preconditioner choice, b and x_0 and nothing else (the variants take
 * exactly the inputs of HS-CG, Section 1).
 *
 * Variants (one fused CUDA sweep per grid-wide reduction):
 *   PRCG_HS       HS-CG, Algorithm 1 -- two reductions per iteration
 *   PRCG_PR       PR-CG, Algorithm 2 -- nu'_k predicted by Eq. 2.3, nu_k
 *                 recomputed with mu, sigma, gamma in one reduction
 *   PRCG_PIPE_PR  pipe-PR-CG, Algorithm 3 -- s, s~ from the predicted w',
 *                 u = A s~ and w = A r~ (recomputed) in one pass over A
 *                 together with the four inner products
 *   PRCG_M, PRCG_PIPE_M, PRCG_CGCG, PRCG_GV are the Appendix E variants
 *                 (M-CG, pipe-PR-M-CG, Chronopoulos-Gear CG in 2 sweeps,
 *                 Ghysels-Vanroose pipelined CG in 1 sweep per iteration).
 *   PRCG_PR_NO_RECOMPUTE, PRCG_PIPE_PR_NO_RECOMPUTE are the ablations the
 *                 paper's analysis compares against: PR-CG whose scalar
 *                 recurrences continue from the predicted nu'_k instead of
 *                 the recomputed nu_k (Section 3.1, Fig. 1; nu' may turn
 *                 negative once ||r_k|| ~ sqrt(eps), which reports
 *                 PRCG_BREAKDOWN), and pipe-PR-CG that carries w_k = w'_k
 *                 instead of recomputing A r~_k (Section 3.2, Fig. 2: the
 *                 w'-gap accumulates).  Same sweeps as PRCG_PR and
 *                 PRCG_PIPE_PR (the pipe ablation forms only u = A s~).
 *
 * Threading: a context is not thread-safe; use one context per host thread.
 * All work of a context runs on the CUDA stream given at creation (or the
 * legacy default stream when NULL) and on one internal stream ordered after it.
 *
 * Pointers: every array argument may be a host pointer (pageable or pinned)
 * or a device pointer of the current device; copies use unified addressing
 * (cudaMemcpyDefault), which tells the two apart.  Nothing passed in is
 * retained after the call returns; the caller keeps ownership.
 *
 * Return values: an int status, PRCG_OK (0) on success.  Negative values
 * mean no result was produced; prcg_last_error() describes the failure.
 */
#ifndef PRCG_H
#define PRCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct prcg_ctx prcg_ctx;

enum prcg_variant {
    PRCG_HS = 0,
    PRCG_PR = 1,
    PRCG_PIPE_PR = 2,
    PRCG_M = 3,
    PRCG_PIPE_M = 4,
    PRCG_CGCG = 5,
    PRCG_GV = 6,
    PRCG_PR_NO_RECOMPUTE = 7,
    PRCG_PIPE_PR_NO_RECOMPUTE = 8
};

enum prcg_precond {
    PRCG_PRECOND_NONE = 0,
    PRCG_PRECOND_JACOBI = 1   /* M^{-1} = diag(1 / a_ii) (Section 4) */
};

enum prcg_status {
    PRCG_OK = 0,               /* ||r_K|| / ||b|| <= tol                         */
    PRCG_NOT_CONVERGED = 1,    /* K = maxit reached; x holds x_maxit            */
    PRCG_BREAKDOWN = 2,        /* mu <= 0, nu <= 0, nu' < 0 or a non-finite
                                  scalar (Section 3.1: the predicted nu' must
                                  stay positive); x holds the last iterate    */
    PRCG_ERR_INVALID = -1,     /* bad argument                                  */
    PRCG_ERR_CUDA = -2,        /* a CUDA call failed                            */
    PRCG_ERR_OOM = -3,         /* device allocation failed                      */
    PRCG_ERR_TIMEOUT = -4,     /* a bounded device wait expired (a grid
                                  barrier of the persistent kernel or a TMA
                                  copy), or the device loop ran more bodies
                                  than maxit allows (internal safety limit)  */
    PRCG_ERR_UNSUPPORTED = -5  /* variant / operator combination not built      */
};

/*
 * prcg_create_csr -- context for a sparse matrix in CSR form.
 *   n        number of rows = columns (1 <= n < 2^31)
 *   nnz      number of stored entries (row_ptr[n] == nnz, nnz < 2^31)
 *   row_ptr  int32[n + 1], non-decreasing, row_ptr[0] == 0
 *   col_idx  int32[nnz], each in [0, n)
 *   vals     double[nnz]
 *   precond  prcg_precond; Jacobi needs every a_ii present and > 0
 *   cuda_stream  cudaStream_t (void*) the context's work is ordered on
 * The arrays are copied into context-owned device memory (the caller may
 * free them afterwards).  Symmetry and definiteness are not checked up
 * front: a non-SPD A shows up as PRCG_BREAKDOWN during prcg_solve.
 * With Jacobi, a diagonal whose entries are all bitwise equal is applied as
 * one scalar d = 1 / a_11 (prcg_jacobi_form reports 1): each product d_i v_i
 * is unchanged, the sweeps stop reading a d vector, and where a recurrence
 * subtracts alpha M^{-1} v the scalar is folded into alpha (the same value
 * up to rounding).  The environment variable PRCG_NO_SCALAR_D=1 keeps the
 * vector form.
 * Returns PRCG_ERR_INVALID for inconsistent sizes or indices out of range.
 */
int prcg_create_csr(prcg_ctx** out, int64_t n, int64_t nnz,
                    const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                    int precond, void* cuda_stream);

/*
 * prcg_create_stencil -- matrix-free structured-grid operator, Dirichlet-0.
 *   dim          2 (5-point) or 3 (7-point); nz is ignored (1) for dim 2
 *   nx, ny, nz   grid sizes, lexicographic order with x fastest
 *   face_coeff   NULL: constant-coefficient Poisson, diagonal 2*dim, off-
 *                diagonal -1.  Otherwise one coefficient c_f > 0 per cell face
 *                including boundary faces, concatenated as x-faces
 *                [nz][ny][nx+1], y-faces [nz][ny+1][nx], (3D) z-faces
 *                [nz+1][ny][nx]; A = sum_f c_f (e_a - e_b)(e_a - e_b)^T with
 *                e_b = 0 on boundary faces.  Copied into the context.
 *   diag_shift   added to the diagonal (>= 0 keeps A SPD)
 *   precond      prcg_precond
 * n = nx*ny*nz must be < 2^31.
 * Arithmetic of the constant-coefficient product: (A v)_i = (2*dim + shift)
 * v_i - S_i, where S_i, the sum of the existing neighbours, is formed exactly
 * in 64-bit fixed point and rounded once (see prcg_test_neighbour_sum), then
 * one FP64 FMA; it differs from an FP64 evaluation in the order of the
 * stencil only in rounding, and is the more accurate of the two.  On the
 * graph path of HS-CG, PR-CG, M-CG and the pipelined variants the product
 * sweeps add the neighbours from block fixed-point copies of the vectors
 * instead (prcg_last_fixed_sweeps), and with an integer diagonal in [1, 8]
 * form the whole row in integers (prcg_int_diagonal).  The variable-coefficient product is an FP64 FMA
 * per entry.
 */
int prcg_create_stencil(prcg_ctx** out, int dim, int64_t nx, int64_t ny, int64_t nz,
                        const double* face_coeff, double diag_shift, int precond,
                        void* cuda_stream);

/*
 * prcg_create_dense -- context for a dense symmetric positive definite A
 * (Section 5 stores its model problem, Eq. 4.1, as a dense matrix so that
 * pipe-PR-CG's two products per iteration cost a full pass over A).
 *   n        1 <= n <= 131072
 *   A        n x n FP64, row-major (for symmetric A also column-major), host
 *            or device; copied into the context (column-major with a
 *            leading dimension rounded up to 32), the caller keeps ownership.
 *            Symmetry is not checked: the library forms A^T v.
 *   precond  PRCG_PRECOND_NONE or PRCG_PRECOND_JACOBI (d_i = 1 / a_ii; a
 *            non-positive diagonal entry gives PRCG_ERR_INVALID)
 * Every product A v is formed by a pre-pass over A in column blocks whose
 * partial sums each row then adds in block order (deterministic for a given
 * n on a given GPU model).  Solves with n <= 4096 run as the persistent
 * kernel of prcg_solve; larger ones as the graph with a product kernel
 * before each product sweep.  All seven variants are supported;
 * prcg_solve_f32_refined returns PRCG_ERR_UNSUPPORTED.
 * Returns PRCG_OK, PRCG_ERR_INVALID, PRCG_ERR_OOM or PRCG_ERR_CUDA.
 */
int prcg_create_dense(prcg_ctx** out, int64_t n, const double* A, int precond, void* cuda_stream);

/*
 * prcg_solve -- run one variant from x_0 until ||r_k|| / ||b|| <= tol.
 *   variant   prcg_variant
 *   b         double[n] right-hand side (host or device)
 *   x         double[n]; in: x_0, out: x_K (host or device)
 *   tol       relative tolerance on the updated residual r_k (>= 0)
 *   maxit     maximum number of iterations (>= 0)
 *   residual_history  NULL or double[maxit + 1]; entries 0..K receive
 *             ||r_k|| / ||b|| (updated residual), the rest are untouched
 *   iters_out NULL or receives K, the number of completed iterations
 *   final_true_relres_out NULL or receives ||b - A x_K|| / ||b||
 * Returns PRCG_OK, PRCG_NOT_CONVERGED, PRCG_BREAKDOWN (x holds x_K in all
 * three) or a negative error (x untouched).  If b == 0, x is set to 0 and
 * K = 0.  The call blocks until the result is on the host.
 * Execution: for n <= 2^21 (dense contexts: n <= 4096; the environment
 * variable PRCG_PERSIST_MAX lowers the bound) every variant but the two
 * ablations runs as one persistent cooperative kernel (grid barriers
 * instead of kernel boundaries); larger systems, and the ablations at every
 * size, run as one CUDA graph launch with a device-side while loop.
 */
int prcg_solve(prcg_ctx* ctx, int variant, const double* b, double* x,
               double tol, int maxit, double* residual_history,
               int* iters_out, double* final_true_relres_out);

/*
 * prcg_solve_f32_refined -- FP32 PR-CG inner solves inside FP64 iterative
 * refinement (an extension; the paper's experiments are all FP64).
 * Outer step j: t = b - A x_j in FP64; stop when ||t|| / ||b|| <= tol;
 * otherwise solve A d = t / ||t|| by PR-CG (Algorithm 2) with FP32 vectors
 * and FP32 matrix values to ||r|| <= max(inner_tol, min(0.5, tol / (4 ||t||
 * / ||b||))) -- the last steps stop as soon as tol is within reach -- or
 * inner_maxit iterations,
 * inner products accumulated with compensated FP32 per thread and FP64
 * across threads, alpha / beta / nu' recurrences in FP64; then
 * x_{j+1} = x_j + ||t|| d in FP64.  The run also stops when an outer step
 * does not reduce the true residual.
 *   b, x            as prcg_solve (x: in x_0, out the refined solution)
 *   tol             on the FP64 true residual ||b - A x|| / ||b||
 *   max_outer       refinement steps (>= 0)
 *   inner_tol       relative, in (0, 1); inner_maxit >= 1
 *   outer_out, inner_total_out   NULL or the counts
 *   final_true_relres_out        NULL or ||b - A x|| / ||b|| at return
 *   outer_history   NULL or double[max_outer + 1]: true residual per step
 * Returns PRCG_OK, PRCG_NOT_CONVERGED (max_outer reached or no progress),
 * PRCG_BREAKDOWN (an inner solve made no iteration) or a negative error;
 * PRCG_ERR_UNSUPPORTED for a context that kept the plain CSR layout.
 * prcg_last_timing reports the whole solve as loop_ms.
 */
int prcg_solve_f32_refined(prcg_ctx* ctx, const double* b, double* x, double tol, int max_outer,
                           double inner_tol, int inner_maxit, int* outer_out,
                           int* inner_total_out, double* final_true_relres_out,
                           double* outer_history);

/* ------------------------------------------------------------------------
 * Adjoint gradients (an extension for differentiable use; the paper has no
 * gradients).  For x = A^{-1} b and a loss L(x), with lambda = A^{-1} dL/dx
 * (A is symmetric, so this is a second prcg_solve on the same context):
 * dL/db = lambda and dL/dA = -lambda x^T on the stored entries.
 * ------------------------------------------------------------------------ */

/* Replace the face coefficients (same grid and layout as at creation) and the
 * diagonal shift of a variable-coefficient stencil context; the diagonal and
 * the Jacobi vector are recomputed. */
int prcg_update_faces(prcg_ctx* ctx, const double* face_coeff, double diag_shift);

/* grad_faces[f] = -(lambda_a - lambda_b)(x_a - x_b) for the interior face f
 * between cells a and b, -lambda_a x_a for a boundary face of cell a, in the
 * face layout of prcg_create_stencil.  lambda, x: double[n]; all host or
 * device. */
int prcg_grad_faces(prcg_ctx* ctx, const double* lambda, const double* x, double* grad_faces);

/* grad_vals[e] = -lambda_i x_{col_idx[e]} for every stored entry e of row i,
 * in the caller's CSR order (CSR contexts only). */
int prcg_grad_csr_values(prcg_ctx* ctx, const double* lambda, const double* x, double* grad_vals);

/*
 * prcg_last_timing -- device time of the last prcg_solve on this context,
 * measured with CUDA events around its phases on the context's stream:
 *   init_ms   initialisation (r_0 ... first reduction)
 *   loop_ms   the iteration loop (all K iterations, including the device-
 *             side loop control)
 *   iters     K
 * Any pointer may be NULL.
 */
int prcg_last_timing(const prcg_ctx* ctx, float* init_ms, float* loop_ms, int* iters);

/*
 * prcg_time_sweeps -- average device time of each sweep (kernel) of one
 * iteration of `variant`, from CUDA events recorded around every launch on
 * the context's stream.  Runs initialize(), two untimed iterations (after
 * which every sweep is in the form it takes for the rest of a solve) and
 * then `reps` timed iterations for a fixed right-hand side without
 * structure (b_i in [0.5, 1.5), a hash of i) and x_0 = 0, with the stopping
 * and breakdown tests switched off (the
 * sweeps always do their full work), and leaves the context's vectors in an
 * unspecified state (the next prcg_solve copies its own b and x_0 in).
 *   ms_per_sweep  float[3]: HS: sweeps A (x, r), B (p), C (s = A p);
 *                 PR / M: A (x, r, r~, p), B (s = A p and the inner products);
 *                 CG-CG: A (p, s, x, r, r~), B (w = A r~ and the inner
 *                 products); pipe-PR / pipe-M / GV: the single sweep.  For a
 *                 dense context a product sweep's time includes its product
 *                 kernel.  The sweeps are those of the graph path.
 *   nsweeps       receives the number of sweeps written (3, 2 or 1)
 * The two ablation variants are not timed (PRCG_ERR_UNSUPPORTED).
 */
int prcg_time_sweeps(prcg_ctx* ctx, int variant, int reps, float* ms_per_sweep, int* nsweeps);

/*
 * prcg_last_launches -- number of this library's kernels the last
 * prcg_solve launched: 1 for a persistent solve (plus the optional
 * true-residual sweep); otherwise the initialisation sweeps, the iteration
 * sweeps including the no-op sweeps after convergence within the last loop
 * body, the loop-control kernels, a dense context's product kernels, and
 * the optional true-residual sweep.
 */
int prcg_last_launches(const prcg_ctx* ctx, int64_t* kernels);

/*
 * prcg_last_fixed_sweeps -- how many product sweeps (s = A p) of the last
 * prcg_solve read the block fixed-point copy of p.  On a constant-
 * coefficient stencil the graph path of HS-CG and PR-CG / M-CG stores, in
 * the sweep that forms p, P_i = round(p_i 2^S) as a 64-bit integer with one
 * scale S per vector, chosen from upper bounds of the vectors p is formed
 * from so that every |P_i| < 2^58; the product sweep then adds the 2*dim
 * neighbour values with integer adds and rounds the sum once to FP64.  The
 * error of the neighbour sum is at most 2^-(S+1) per term plus that one
 * rounding: a normwise bound, below 2^-58 max |p| per term, instead of the
 * per-row bound of the fixed-point sum of the other sweeps.  A value
 * outside its window (never expected) makes that sweep use the per-row
 * sums; PRCG_NO_FIXED_P=1 disables the copy.  pipe-PR-CG and pipe-M-CG do
 * the same with copies of r~ and s~ (stored by each sweep, read from the
 * third sweep on) for both of their products; their count is of the sweeps
 * that read them.  0 for the persistent path, the no-recompute ablations
 * and other operators and variants.
 */
int prcg_last_fixed_sweeps(const prcg_ctx* ctx, int64_t* sweeps);

/* prcg_destroy -- free the context and everything it owns; NULL is a no-op. */
/*
 * prcg_jacobi_form -- how the context applies its preconditioner:
 * 0 none, 1 a scalar d (constant stencils, or a CSR / dense diagonal whose
 * entries are all equal), 2 a vector d.  Negative on a NULL context.
 */
int prcg_jacobi_form(const prcg_ctx* ctx);

/*
 * prcg_int_diagonal -- the diagonal c of a constant-coefficient stencil
 * context when it is an integer in [1, 8] (2*dim plus an integer shift, e.g.
 * Poisson: 4 in 2D, 6 in 3D), with which the product sweeps that read a
 * block fixed-point copy P form each row c P_i - sum_j P_j exactly in
 * 64-bit integers and round it once (no FP64 instruction; the error is that
 * of the copy, normwise, see prcg_last_fixed_sweeps).  0 when the diagonal
 * is not such an integer, the operator is not a constant stencil, or
 * PRCG_NO_INT_DIAG=1 was set when the context was created (the row is then
 * the FP64 FMA c p_i - sum).  Negative on a NULL context.
 */
int prcg_int_diagonal(const prcg_ctx* ctx);

int prcg_destroy(prcg_ctx* ctx);

/*
 * prcg_last_error -- message describing the last failure on ctx (or of the
 * last failed create when ctx is NULL).  Valid until the next call on ctx.
 */
const char* prcg_last_error(const prcg_ctx* ctx);

/* prcg_n -- the number of unknowns of the context (or -1 for NULL). */
int64_t prcg_n(const prcg_ctx* ctx);

/*
 * prcg_inject_barrier_skip -- failure injection for tests: in the next
 * prcg_solve that runs as the persistent kernel, CTA `cta` does not arrive
 * at grid barrier number `barrier` (0 = the first of the solve), and every
 * barrier wait gives up after `spin_limit` polls (>= 1024) instead of the
 * default 2^22.  All CTAs then stop at that barrier, the solve returns
 * PRCG_ERR_TIMEOUT with x untouched, and the context stays usable.  Nothing
 * faults or hangs: every wait in the kernel is bounded.  One-shot; the paper
 * has no counterpart.
 */
int prcg_inject_barrier_skip(prcg_ctx* ctx, int cta, int barrier, int64_t spin_limit);

/*
 * prcg_check_guards -- count corrupted guard words.  Every vector, partial
 * sum buffer and scratch array of the context is followed by a 256-byte
 * guard band (its rounding up to a multiple of 32 entries included; the
 * vector pool also starts with one) holding a signalling-NaN bit pattern,
 * which FP64 arithmetic never produces.  A kernel writing past the end of
 * any of them changes a guard word.  *corrupted_out receives the number of
 * changed words (0 when every access stayed in bounds).  A test utility in
 * place of a memory checker; the paper has no counterpart.  Returns PRCG_OK
 * or a negative error; blocks until the count is on the host.
 */
int prcg_check_guards(prcg_ctx* ctx, int64_t* corrupted_out);

/*
 * prcg_test_neighbour_sum -- run the constant-coefficient stencil's
 * neighbour sum on the device for count tuples of `terms` doubles (4: the
 * 2D 5-point stencil, 6: the 3D 7-point stencil), for tests of that kernel
 * arithmetic.  The sum is formed in 64-bit fixed point aligned to the
 * largest term and rounded once to nearest-even (error at most one rounding
 * of the exact sum plus terms * 2^-59 times the largest term); tuples with a
 * non-finite term, a term of magnitude >= 2^1018, or all terms below 2^-959
 * are added in sequential FP64 instead, so NaN and infinity propagate.
 *   v     host or device, count x terms doubles, tuple-major
 *   out   host or device, count doubles
 * Returns PRCG_OK, PRCG_ERR_INVALID (terms not 4 or 6, count < 0, NULL
 * arrays) or a CUDA error; prcg_last_error(NULL) describes a failure.
 * Blocks until out is written; allocates and frees its own device buffers.
 */
int prcg_test_neighbour_sum(int terms, const double* v, int64_t count, double* out);

/*
 * prcg_trace_enable -- record, during every later prcg_solve on ctx (on != 0)
 * or no more (on == 0), the scalars each iteration forms.  Costs a few
 * device stores per iteration and a buffer of (maxit + 2) x 10 doubles.
 *
 * prcg_trace_get -- copy the trace of the last solve to out (host or device,
 * slots x 10 doubles); returns the number of slots copied (<= slots; K + 1
 * after a solve of K iterations) or a negative error.  Slot k, fields in
 * order: alpha_{k-1} (the step length applied in iteration k), beta_k,
 * nu_k, nu'_k (the predicted nu of Eq. 2.3 / Meurant's form), mu_k,
 * sigma_k, gamma_k, rho_k = <r_k, r_k>, eta_k (CG-CG, GV-CG), unused.
 * Slot 0 holds initialize()'s nu_0, mu_0, sigma_0, gamma_0, rho_0.  Fields a
 * variant does not form are NaN, and so are those of slot K that follow the
 * stopping test (beta_K, mu_K of HS-CG, for instance).  The paper has no
 * counterpart: this exposes the quantities its analysis (Section 3) reasons
 * about, for tests and studies.
 */
int prcg_trace_enable(prcg_ctx* ctx, int on);
int prcg_trace_get(prcg_ctx* ctx, double* out, int slots);

/*
 * prcg_error_anorm -- the A-norm of the error, ||x* - x||_A =
 * sqrt((x* - x)^T A (x* - x)), with the context's operator A (not the
 * preconditioned one).  This is the error measure of the paper's
 * convergence study (Section 4: iterations to reduce it by a factor 10^5,
 * and its minimum over the run, Table 2).
 *   x_star, x  length n, host or device (FP64); read only, borrowed
 *   err_out    host double, receives the norm (a negative e^T A e from
 *              rounding is reported as 0)
 * Returns PRCG_OK or a negative error.  Uses the context's scratch vectors,
 * so it must not overlap a prcg_solve on the same context; blocks until the
 * value is on the host.
 */
int prcg_error_anorm(prcg_ctx* ctx, const double* x_star, const double* x, double* err_out);

/* ------------------------------------------------------------------------
 * Batched solver: many independent SPD systems of uneven size in one launch.
 *
 * Each system i is the 2D 5-point operator of prcg_create_stencil (face_coeff
 * NULL) on an nx[i] x ny[i] grid with diagonal shift shift[i] >= 0.  One
 * persistent kernel (captured in a CUDA graph with the reset of its work
 * queue) solves all of them with PR-CG (Algorithm 2): each thread-block
 * cluster takes the next system from a device queue ordered by estimated
 * cost (n * sqrt(condition number), largest first) and iterates it to
 * ||r_k|| / ||b|| <= tol with cluster-wide reductions in distributed shared
 * memory.  Cluster and CTA sizes come from prcg_batched_configure (the
 * Python autotuner picks them); the default is 1 CTA of 256 threads.
 * ------------------------------------------------------------------------ */
typedef struct prcg_batch prcg_batch;

/* nx, ny, shift: host arrays of nsys entries (copied).  precond as above
 * (Jacobi is the scalar 1 / (4 + shift[i])).  n_i = nx[i]*ny[i] < 2^30. */
int prcg_batched_create(prcg_batch** out, int nsys, const int32_t* nx, const int32_t* ny,
                        const double* shift, int precond, void* cuda_stream);

/* cluster in {1, 2, 4, 8, 16} CTAs, threads per CTA a multiple of 32 in
 * [64, 1024]; PRCG_ERR_UNSUPPORTED if the cluster cannot be resident. */
int prcg_batched_configure(prcg_batch* bt, int cluster, int threads);

/* Split launch: the nbig systems of largest estimated cost (1 <= nbig < nsys)
 * are solved by one persistent launch with clusters of cluster_big CTAs x
 * threads_big (one cluster per system, the first launch placed with the
 * highest stream priority), the others by a second persistent launch of
 * cluster_rest x threads_rest sized to the residency the first leaves free;
 * the two run side by side in the solve's graph, each with its own work
 * queue (no kernel waits on the other).  Large systems then get more SMs
 * without slowing the many small ones.  Same limits as
 * prcg_batched_configure; prcg_batched_configure returns to one launch. */
int prcg_batched_configure_split(prcg_batch* bt, int nbig, int cluster_big, int threads_big,
                                 int cluster_rest, int threads_rest);

/* b, x: sum(n_i) doubles each, systems concatenated in creation order (host or
 * device); x holds x_0 on entry and x_K per system on return.  iters_out,
 * status_out (int32[nsys]) and true_relres_out (double[nsys], ||b - A x|| /
 * ||b|| per system) may be NULL.  Returns the worst per-system status
 * (PRCG_OK < PRCG_NOT_CONVERGED < PRCG_BREAKDOWN) or a negative error. */
int prcg_batched_solve(prcg_batch* bt, const double* b, double* x, double tol, int maxit,
                       int32_t* iters_out, int32_t* status_out, double* true_relres_out);

/* device time (CUDA events) of the last batched solve's graph launch */
int prcg_batched_last_ms(const prcg_batch* bt, float* ms);

/* the launch configuration in use: cluster size, CTA size, resident clusters
 * (of the first launch when split) */
int prcg_batched_config(const prcg_batch* bt, int* cluster, int* threads, int* clusters);

/* the split in use: nbig and the second launch's cluster size, CTA size and
 * clusters (all 0 for a single launch); any pointer may be NULL */
int prcg_batched_split(const prcg_batch* bt, int* nbig, int* cluster_rest, int* threads_rest,
                       int* clusters_rest);

const char* prcg_batched_last_error(const prcg_batch* bt);

int prcg_batched_destroy(prcg_batch* bt);

/*
 * prcg_pr_solve_stencil_noalloc -- PR-CG on a small constant-coefficient
 * stencil system without any device allocation.  The paper has no
 * counterpart: this is a deployment form of the PR-CG sweep for callers that
 * cannot allocate device memory -- code running under another framework's
 * memory pool or allocator hooks, real-time loops that forbid cudaMalloc /
 * cudaFree after start-up, and callers that cannot keep a context alive.
 *
 * The operator is the one of prcg_create_stencil with face_coeff == NULL
 * (diagonal 2*dim + diag_shift, off-diagonal -1, Dirichlet-0).  The whole
 * solve runs as one single-CTA kernel; the iteration vectors live in a
 * file-scope device array of fixed size, allocated when the library is
 * loaded and kept by every GPU that loads it until the process exits:
 * n = nx*ny*nz must be <= 65536 (the array holds 8 vectors of 65536 doubles,
 * 4 MiB).  Larger n returns PRCG_ERR_INVALID.
 *   b, x              device pointers the caller owns (x: in x_0, out x_K),
 *                     in memory of the current device (or managed memory);
 *                     another GPU's memory returns PRCG_ERR_INVALID
 *   tol, maxit        as prcg_solve; the solve is one kernel that cannot be
 *                     interrupted, so maxit must be <= 4 n + 1000 (larger
 *                     returns PRCG_ERR_INVALID): a tolerance the system cannot
 *                     reach then ends with PRCG_NOT_CONVERGED in bounded time
 *   residual_history  NULL or device double[maxit + 1] (current device)
 *   iters_out         NULL or receives K
 *   cuda_stream       stream to run on (NULL: legacy default stream)
 * b == 0 gives x = 0 with K = 0, as prcg_solve does.
 * Returns PRCG_OK / PRCG_NOT_CONVERGED / PRCG_BREAKDOWN or a negative error.
 * Blocks until the result is known.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress): make that first call
 * before any stream capture.  That set-up is safe when several host threads
 * make their first call at once.  All calls share the one array, so calls
 * that overlap on the GPU (other streams or host threads) race with each
 * other and must be serialised by the caller.
 */
int prcg_pr_solve_stencil_noalloc(int dim, int64_t nx, int64_t ny, int64_t nz,
                                  double diag_shift, int precond, const double* b, double* x,
                                  double tol, int maxit, double* residual_history,
                                  int* iters_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PRCG_H */
