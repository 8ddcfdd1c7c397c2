/*
 * Multi-threaded C oracle of HS-CG, PR-CG and pipe-PR-CG on a CSR matrix.
 *
 * TEST INFRASTRUCTURE ONLY.  It exists so that the CPU baseline of the
 * benchmark runs the method on every host core; only the tests and the
 * CPU legs of bench.py load it (through oracle/c_oracle.py).  The CUDA
 * library shares no code with it.
 *
 * Each variant follows the paper's algorithm step by step, one loop per
 * vector operation and one per inner product, in the order and notation of
 *   HS-CG       Algorithm 1
 *   PR-CG       Algorithm 2 (nu'_k by Eq. 2.3)
 *   pipe-PR-CG  Algorithm 3 (the s, s~, w, w~ recurrences of Section 2.2)
 * with initialize() of Appendix E in dependency order.  Arithmetic is plain
 * FP64 (compiled with -ffp-contract=off, so no fused multiply-add).  Every
 * loop is an OpenMP parallel loop; an inner product is an OpenMP sum
 * reduction ("plain-dot" mode: its summation order depends on the thread
 * count, so runs with different thread counts differ in rounding).
 *
 * Readings shared with the numpy oracle (oracle/cg_variants.py): stop at the
 * first k with ||r_k|| / ||b|| <= tol on the updated residual (rho_k =
 * <r_k, r_k>, an extra inner product with a preconditioner); the scalars of
 * iteration k are formed at its start (Section 2.2.1) and a breakdown there
 * (mu <= 0, nu < 0, nu' < 0, nu == 0 or a non-finite scalar; Section 3.1)
 * returns x_{k-1} with K = k - 1; M^{-1} = diag(d).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include <omp.h>

enum { CGO_OK = 0, CGO_NOT_CONVERGED = 1, CGO_BREAKDOWN = 2, CGO_ERR = -1 };
enum { CGO_HS = 0, CGO_PR = 1, CGO_PIPE_PR = 2 };

typedef struct {
  int n;
  const int32_t* rp;
  const int32_t* ci;
  const double* va;
  const double* d;   /* NULL: no preconditioner */
} Sys;

static double now_s(void) {
  struct timespec t;
  clock_gettime(CLOCK_MONOTONIC, &t);
  return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}

/* y = A v */
static void matvec(const Sys* A, const double* v, double* y) {
  const int n = A->n;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int e = A->rp[i]; e < A->rp[i + 1]; ++e) acc += A->va[e] * v[A->ci[e]];
    y[i] = acc;
  }
}

/* y = M^{-1} v (a copy without a preconditioner) */
static void minv(const Sys* A, const double* v, double* y) {
  const int n = A->n;
  if (A->d) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) y[i] = A->d[i] * v[i];
  } else {
    memcpy(y, v, (size_t)n * sizeof(double));
  }
}

static double dot(int n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* y = y + a v */
static void axpy(int n, double a, const double* v, double* y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) y[i] = y[i] + a * v[i];
}

/* y = v + b y */
static void xpby(int n, const double* v, double b, double* y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) y[i] = v[i] + b * y[i];
}

/* y = v - a u */
static void sub_scaled(int n, const double* v, double a, const double* u, double* y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) y[i] = v[i] - a * u[i];
}

static int finite_pos(double v) { return isfinite(v) && v > 0.0; }

typedef struct {
  double tol2bn2;   /* tol^2 ||b||^2 */
  double bnorm;
  int maxit;
  double* hist;     /* ||r_k|| / ||b||, or NULL */
} Run;

/* the stopping test of iteration k on rho_k = <r_k, r_k> */
static int stop_test(const Run* R, int k, double rho) {
  if (R->hist) R->hist[k] = R->bnorm != 0.0 ? sqrt(rho) / R->bnorm : 0.0;
  return rho <= R->tol2bn2;
}

/*
 * cgo_solve -- run one variant; x holds x_0 on entry and x_K on return.
 * Returns the status; *iters = K; *init_s and *loop_s receive the wall time
 * of initialize() and of the iteration loop.  threads <= 0 keeps OpenMP's
 * default.
 */
int cgo_solve(int variant, int n, const int32_t* rp, const int32_t* ci, const double* va,
              const double* d, const double* b, double* x, double tol, int maxit, int threads,
              int* iters, double* hist, double* init_s, double* loop_s) {
  if (n < 1 || !rp || !ci || !va || !b || !x || !iters || maxit < 0 || !(tol >= 0.0)) return CGO_ERR;
  if (variant < CGO_HS || variant > CGO_PIPE_PR) return CGO_ERR;
  if (threads > 0) omp_set_num_threads(threads);
  const Sys A = {n, rp, ci, va, d};
  const int pc = d != NULL;
  const size_t V = (size_t)n * sizeof(double);
  double* r = malloc(V);
  double* rt = malloc(V);
  double* p = malloc(V);
  double* s = malloc(V);
  double* st = malloc(V);
  double* w = malloc(V);
  double* wt = malloc(V);
  double* u = malloc(V);
  double* ut = malloc(V);
  double* t = malloc(V);
  if (!r || !rt || !p || !s || !st || !w || !wt || !u || !ut || !t) {
    free(r); free(rt); free(p); free(s); free(st); free(w); free(wt); free(u); free(ut); free(t);
    return CGO_ERR;
  }
  const double t0 = now_s();
  /* initialize() (Appendix E), dependency order */
  matvec(&A, x, t);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) r[i] = b[i] - t[i];                 /* r_0 = b - A x_0 */
  minv(&A, r, rt);                                                 /* r~_0 = M^{-1} r_0 */
  double nu = dot(n, r, rt);                                       /* nu_0 */
  memcpy(p, rt, V);                                                /* p_0 = r~_0 */
  matvec(&A, p, s);                                                /* s_0 = A p_0 */
  double mu = dot(n, p, s);                                        /* mu_0 */
  minv(&A, s, st);                                                 /* s~_0 */
  double sigma = dot(n, rt, s);                                    /* sigma_0 */
  double gamma = dot(n, st, s);                                    /* gamma_0 */
  if (variant == CGO_PIPE_PR) {
    matvec(&A, rt, w);                                             /* w_0 = A r~_0 */
    minv(&A, w, wt);                                               /* w~_0 */
    matvec(&A, st, u);                                             /* u_0 = A s~_0 */
    minv(&A, u, ut);                                               /* u~_0 */
  }
  const double bn2 = dot(n, b, b);
  Run R = {tol * tol * bn2, sqrt(bn2), maxit, hist};
  const double rho0 = dot(n, r, r);
  const double t1 = now_s();
  int status = CGO_NOT_CONVERGED, K = maxit;
  if (bn2 == 0.0 || stop_test(&R, 0, rho0)) {
    status = CGO_OK;
    K = 0;
    goto done;
  }
  for (int k = 1; k <= maxit; ++k) {
    if (variant == CGO_HS) {
      if (!isfinite(nu) || !finite_pos(mu) || nu < 0.0) { status = CGO_BREAKDOWN; K = k - 1; break; }
      const double alpha = nu / mu;                                /* alpha_{k-1} */
      axpy(n, alpha, p, x);                                        /* x_k */
      axpy(n, -alpha, s, r);                                       /* r_k */
      minv(&A, r, rt);                                             /* r~_k = M^{-1} r_k */
      const double nun = dot(n, rt, r);                            /* nu_k */
      const double rho = pc ? dot(n, r, r) : nun;
      if (stop_test(&R, k, rho)) { status = CGO_OK; K = k; break; }
      if (!finite_pos(nun)) { status = CGO_BREAKDOWN; K = k; break; }
      const double beta = nun / nu;                                /* beta_k */
      xpby(n, rt, beta, p);                                        /* p_k = r~_k + beta_k p_{k-1} */
      matvec(&A, p, s);                                            /* s_k = A p_k */
      mu = dot(n, p, s);                                           /* mu_k */
      nu = nun;
    } else {
      if (!isfinite(nu) || !finite_pos(mu) || nu < 0.0) { status = CGO_BREAKDOWN; K = k - 1; break; }
      const double alpha = nu / mu;                                /* alpha_{k-1} */
      const double nup = nu - 2.0 * alpha * sigma + alpha * alpha * gamma;   /* Eq. 2.3 */
      if (!isfinite(nup) || nup < 0.0 || nu == 0.0) { status = CGO_BREAKDOWN; K = k - 1; break; }
      const double beta = nup / nu;                                /* beta_k */
      axpy(n, alpha, p, x);                                        /* x_k */
      axpy(n, -alpha, s, r);                                       /* r_k */
      if (pc) axpy(n, -alpha, st, rt);                             /* r~_k by recurrence */
      const double* rtk = pc ? rt : r;
      if (variant == CGO_PR) {
        xpby(n, rtk, beta, p);                                     /* p_k */
        matvec(&A, p, s);                                          /* s_k = A p_k */
        minv(&A, s, st);                                           /* s~_k */
      } else {
        sub_scaled(n, w, alpha, u, w);                             /* w'_k = w_{k-1} - alpha u_{k-1} */
        if (pc) sub_scaled(n, wt, alpha, ut, wt);                  /* w~'_k */
        xpby(n, rtk, beta, p);                                     /* p_k */
        xpby(n, w, beta, s);                                       /* s_k = w'_k + beta s_{k-1} */
        if (pc) xpby(n, wt, beta, st);                             /* s~_k = w~'_k + beta s~_{k-1} */
        else memcpy(st, s, V);
        matvec(&A, st, u);                                         /* u_k = A s~_k */
        minv(&A, u, ut);                                           /* u~_k */
        matvec(&A, rtk, w);                                        /* w_k = A r~_k (recomputed) */
        minv(&A, w, wt);                                           /* w~_k */
      }
      mu = dot(n, p, s);                                           /* mu_k */
      sigma = dot(n, rtk, s);                                      /* sigma_k */
      gamma = dot(n, st, s);                                       /* gamma_k */
      nu = dot(n, rtk, r);                                         /* nu_k (recomputed) */
      const double rho = pc ? dot(n, r, r) : nu;
      if (stop_test(&R, k, rho)) { status = CGO_OK; K = k; break; }
    }
  }
done:;
  const double t2 = now_s();
  *iters = K;
  if (init_s) *init_s = t1 - t0;
  if (loop_s) *loop_s = t2 - t1;
  free(r); free(rt); free(p); free(s); free(st); free(w); free(wt); free(u); free(ut); free(t);
  return status;
}

/* the number of threads OpenMP runs a parallel region with */
int cgo_max_threads(void) { return omp_get_max_threads(); }
