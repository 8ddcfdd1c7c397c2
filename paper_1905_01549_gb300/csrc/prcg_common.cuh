// Shared device-side definitions of the predict-and-recompute CG library:
// the device-resident scalar block, the plan of device pointers every
// kernel receives, and the deterministic two-level grid reduction that
// replaces the paper's global reduction (Table 1, C_gr).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "prcg_reduce.cuh"

namespace prcg {

constexpr int kBlock = 256;             // threads per CTA for every sweep
constexpr int kMaxGrid = 152 * 16;      // upper bound of CTAs of one sweep
constexpr int kMaxNV = 8;               // doubles reduced per CTA
constexpr int kRunning = -100;          // status while the loop runs

enum Variant {
  V_HS = 0, V_PR = 1, V_PIPE = 2, V_M = 3, V_PIPE_M = 4, V_CGCG = 5, V_GV = 6,
  // the no-recompute ablations: PR-CG with nu_k carried as nu'_k (Section 3.1,
  // Fig. 1) and pipe-PR-CG with w_k carried as w'_k (Section 3.2, Fig. 2)
  V_PR_NR = 7, V_PIPE_NR = 8
};

// Device-resident scalar block (one per context).  Written by the last CTA
// of each sweep after the grid reduction, read by every CTA of the next.
struct DevState {
  // values of the latest reduction
  double nu, mu, sigma, gamma, rho, eta;
  // scalars of the next vector sweep (Section 2.2.1: formed up front)
  double alpha, beta, nu_pred;
  double bnorm2;
  // per-solve parameters
  double tol;
  double tol2;           // tol^2: the stopping test compares squared norms
  double* hist;          // device array, >= maxit + 1 entries
  int maxit;
  int maxbodies;         // safety limit for the device-side while loop
  // loop state
  int k;                 // completed iterations
  int status;            // kRunning until decided
  int done;              // 1 once status is decided: every later sweep is a no-op
  int zero_rhs;          // b == 0: the result is x = 0
  unsigned arrive;       // CTAs that finished the current sweep
  unsigned bodies;       // executions of the while-loop body
  int profile;           // timing runs: never finish, keep every sweep doing its work
  double arg;            // mixed precision: 1 / ||t|| of the current refinement step
  double* trace;         // optional scalar trace, (maxit + 2) x kTraceFields, or NULL
  int carry_nu;          // 1: nu_k := nu'_k for k >= 1 (the PR-CG ablation of Fig. 1)
  // Block fixed-point copy of p for the constant-stencil product sweeps of
  // HS-CG and PR-CG (prcg_isum.cuh, to_fixed): the scale of the next copy
  // is chosen from bounds of the magnitudes of the vectors that form p.
  int pf_allow;          // set by the host: 0 keeps the per-row fixed-point sums
  int pf_on;             // the sweep that forms p also stores its fixed-point copy
  int pf_scale;          // S of that copy: P_i = round(p_i 2^S)
  int pf_bad;            // a value of the copy did not fit its window (fall back)
  unsigned amax_r, amax_p, amax_s;   // high words (sign cleared) of max |r~|, |p|, |s|
  int pf_sweeps;         // product sweeps of this solve that read the fixed-point copy
  // pipe-PR-CG on a constant stencil: block fixed-point copies of r~ and s~
  // per buffer q.  pq_on[q]: the sweep that writes buffer q also stores the
  // copies, with scales pq_scale_r[q], pq_scale_s[q]; pq_bad[q]: a value did
  // not fit its window.  The sweep that reads buffer q uses the copies when
  // pq_on[q] && !pq_bad[q].
  int pq_on[2], pq_bad[2];
  int pq_scale_r[2], pq_scale_s[2];
};

// Scalar trace: slot k holds the scalars of iteration k in the oracle's
// convention -- alpha_{k-1} (applied in iteration k), beta_k, nu_k, nu'_k,
// mu_k, sigma_k, gamma_k, rho_k = <r_k, r_k>, eta_k -- slot 0 those of
// initialize().  Unset fields keep the host's fill (NaN).
enum TraceField {
  TR_ALPHA = 0, TR_BETA, TR_NU, TR_NU_PRED, TR_MU, TR_SIGMA, TR_GAMMA, TR_RHO, TR_ETA,
  kTraceFields = 10
};

__device__ __forceinline__ void trace(const DevState* S, int k, int f, double v) {
  double* t = S->trace;
  if (t && k >= 0 && k <= S->maxit + 1) t[(size_t)k * kTraceFields + f] = v;
}

// Pointers of one context; kernels take what they need by value.
struct Vecs {
  double* x;
  const double* b;
  double* r[2];
  double* rt[2];
  double* p[2];
  double* s[2];
  double* st[2];
  double* w[2];
  double* u[2];
  double* t;             // scratch vector (true residual, GV's t_k)
  long long* pf;         // block fixed-point copy of p (constant stencils)
  long long* rtf[2];     // pipe-PR-CG: fixed-point copies of r~ and s~ per buffer
  long long* stf[2];
};

// FP32 vectors of the mixed-precision inner solve (A d = r in FP32).
struct Vecs32 {
  float* r;
  float* rt;
  float* p;
  float* s;
  float* d;      // the inner iterate (correction)
  float* rhs;    // r_outer / ||r_outer||
};

// Compensated (Kahan) FP32 accumulator: inner products of the FP32 solve
// accumulate their FP32 products without FP64 instructions; the running
// error term keeps the sum accurate to about one FP32 rounding.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ double ldcs(const double* p) { return __ldcs(p); }
__device__ __forceinline__ double ldg(const double* p) { return __ldg(p); }

// Grid-wide sum of v: each CTA writes its partial, the last CTA to arrive
// adds all partials in CTA order (deterministic for a fixed grid) and
// returns true with the totals in tot (thread 0).  No CTA ever waits.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, DevState* S,
                                         double (&tot)[NV]) {
  __shared__ double sm[NV * 32];
  __shared__ int is_last;
  block_sum<NV>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < NV; ++m) partials[blockIdx.x * NV + m] = v[m];
    __threadfence();
    unsigned t = atomicAdd(&S->arrive, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) acc[m] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int m = 0; m < NV; ++m) acc[m] += __ldcg(&partials[b * NV + m]);
  }
  block_sum<NV>(acc, sm, (threadIdx.x & ~31) < (int)gridDim.x);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < NV; ++m) tot[m] = acc[m];
    S->arrive = 0;
  }
  return true;
}

__device__ __forceinline__ bool finite(double v) { return isfinite(v); }

// --------------------------------------------------------------------------
// scalar steps, run by thread 0 of the last CTA of a sweep
// --------------------------------------------------------------------------

// Decide convergence for iteration k from rho_k = <r_k, r_k>; returns true
// (and finishes the run) when ||r_k||^2 <= tol^2 ||b||^2 or k == maxit.
// The history records rho_k; the host converts it to ||r_k|| / ||b|| (a
// square root and a division cost ~1000 cycles of FP64 latency here).
__device__ __forceinline__ bool record_and_test(DevState* S, int k, double rho) {
  S->k = k;
  if (S->profile) return false;
  if (S->hist) S->hist[k] = rho;
  if (rho <= S->tol2 * S->bnorm2) {
    S->status = 0;
    S->done = 1;
    return true;
  }
  if (k >= S->maxit) {
    S->status = 1;
    S->done = 1;
    return true;
  }
  return false;
}

__device__ __forceinline__ void breakdown(DevState* S) {
  if (S->profile) return;
  S->status = 2;
  S->done = 1;
}

// alpha_k = nu_k / mu_k and, for the predict-and-recompute variants,
// nu'_{k+1} (Eq. 2.3, or Meurant's form) and beta_{k+1} = nu'_{k+1} / nu_k.
//
// With carry_nu the recomputed <r~_k, r_k> in S->nu is only recorded: the
// scalar recurrences continue from the predicted nu'_k of the previous step,
// still in S->nu_pred (nu_0 is always the inner product of initialize()).
__device__ __forceinline__ void scalar_step_pr(DevState* S, bool meurant) {
  const double nu = (S->carry_nu && S->k > 0) ? S->nu_pred : S->nu;
  const double mu = S->mu, sigma = S->sigma, gamma = S->gamma;
  if (!finite(nu) || !finite(mu) || !(mu > 0.0) || nu < 0.0) { breakdown(S); return; }
  const double alpha = nu / mu;
  double nu_pred;
  if (meurant) {
    nu_pred = -nu + alpha * alpha * gamma;
  } else {
    nu_pred = nu - 2.0 * alpha * sigma + alpha * alpha * gamma;
  }
  if (!finite(nu_pred) || nu_pred < 0.0 || nu == 0.0) { breakdown(S); return; }
  S->alpha = alpha;
  S->nu_pred = nu_pred;
  S->beta = nu_pred / nu;
  trace(S, S->k + 1, TR_ALPHA, alpha);
  trace(S, S->k + 1, TR_NU_PRED, nu_pred);
  trace(S, S->k + 1, TR_BETA, S->beta);
}

// CTA-wide maximum of v (thread-local values), added to *dst with one
// global atomicMax by thread 0.  Every thread of the CTA must call it.
__device__ __forceinline__ void cta_atomic_max(unsigned v, unsigned* dst) {
  __shared__ unsigned smax;
  if (threadIdx.x == 0) smax = 0u;
  __syncthreads();
  v = __reduce_max_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && v) atomicMax(&smax, v);
  __syncthreads();
  if (threadIdx.x == 0 && smax) atomicMax(dst, smax);
}

// Magnitude key of a double for the max trackers: its high word, sign cleared.
__device__ __forceinline__ unsigned mag_hi(double v) {
  return (unsigned)__double2hiint(v) & 0x7FFFFFFFu;
}

// The reduction of iteration k of PR-CG / pipe-PR-CG (values already in S).
__device__ __forceinline__ void trace_pr_sums(const DevState* S, int k) {
  trace(S, k, TR_NU, S->nu);
  trace(S, k, TR_MU, S->mu);
  trace(S, k, TR_SIGMA, S->sigma);
  trace(S, k, TR_GAMMA, S->gamma);
  trace(S, k, TR_RHO, S->rho);
}

}  // namespace prcg
