// Fused sweeps of HS-CG (Algorithm 1), PR-CG / M-CG (Algorithm 2 and its
// Appendix E variant) and pipe-PR-CG / pipe-PR-M-CG (Algorithm 3).
//
// One sweep = one pass over the rows that does every vector update the
// variant allows before its next global reduction, the matrix-vector
// product(s), the partial inner products, and the grid reduction; the last
// CTA forms the next scalars (Section 2.2.1) on the device.  Vectors that
// other rows gather in the same sweep are double-buffered: the sweep of
// iteration k reads buffer (k-1)&1 and writes buffer k&1.
#pragma once

#include "prcg_ops.cuh"

namespace prcg {

// Rows are processed in tiles of kBlock consecutive rows; CTAs stride over
// tiles so that every CTA's partial sums have a fixed order.
#define PRCG_ROWS(i, n)                                                         \
  for (int tile_ = blockIdx.x; tile_ * kBlock < (n); tile_ += gridDim.x)        \
    for (int i = tile_ * kBlock + threadIdx.x; i < (n) && i < (tile_ + 1) * kBlock; i += kBlock)

// ---------------------------------------------------------------- initialize()
// r_0 = b - A x_0, r~_0 = M^{-1} r_0, p_0 = r~_0; nu_0, <r_0, r_0>, <b, b>.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_init_a(Op op, Pc pc, Vecs V, DevState* S,
                                                   double* partials) {
  if (__ldcg(&S->done)) return;
  double acc[3] = {0.0, 0.0, 0.0};
  const double* __restrict__ x = V.x;
  PRCG_ROWS(i, op.n) {
    const double ax = op.row(i, [&](int j) { return __ldg(x + j); });
    const double bi = __ldg(V.b + i);
    const double r = bi - ax;
    const double rt = Pc::on ? pc(i) * r : r;
    V.r[0][i] = r;
    if (Pc::on) V.rt[0][i] = rt;
    V.p[0][i] = rt;
    acc[0] += rt * r;
    acc[1] += r * r;
    acc[2] += bi * bi;
  }
  double tot[3];
  if (grid_sum<3>(acc, partials, S, tot) && threadIdx.x == 0) {
    S->nu = tot[0];
    S->rho = tot[1];
    S->bnorm2 = tot[2];
    S->k = 0;
    if (tot[2] == 0.0) {
      S->zero_rhs = 1;
      if (S->hist) S->hist[0] = 0.0;
      S->status = 0;
      S->done = 1;
    } else {
      record_and_test(S, 0, tot[1]);
    }
  }
}

// s_0 = A p_0, s~_0 = M^{-1} s_0 (and w_0 = A r~_0, which is the same
// product because p_0 = r~_0); mu_0, sigma_0, gamma_0; then alpha_0 (and
// nu'_1, beta_1 for the predict-and-recompute variants).
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_init_b(Op op, Pc pc, Vecs V, DevState* S,
                                                   double* partials, int variant) {
  if (__ldcg(&S->done)) return;
  const bool pipe = variant == V_PIPE || variant == V_PIPE_M || variant == V_GV;
  double acc[3] = {0.0, 0.0, 0.0};
  const double* __restrict__ p = V.p[0];
  PRCG_ROWS(i, op.n) {
    const double s = op.row(i, [&](int j) { return __ldg(p + j); });
    const double st = Pc::on ? pc(i) * s : s;
    V.s[0][i] = s;
    if (Pc::on) V.st[0][i] = st;
    if (pipe) V.w[0][i] = s;
    const double pi = __ldg(p + i);
    const double rt = Pc::on ? __ldg(V.rt[0] + i) : __ldg(V.r[0] + i);
    acc[0] += pi * s;
    acc[1] += rt * s;
    acc[2] += st * s;
  }
  double tot[3];
  if (grid_sum<3>(acc, partials, S, tot) && threadIdx.x == 0) {
    S->mu = tot[0];
    S->sigma = tot[1];
    S->gamma = tot[2];
    if (variant == V_PR || variant == V_PIPE || variant == V_M || variant == V_PIPE_M) {
      scalar_step_pr(S, variant == V_M || variant == V_PIPE_M);
    } else {
      const double nu = S->nu, mu = tot[0];
      if (!finite(nu) || !finite(mu) || !(mu > 0.0) || nu < 0.0) {
        breakdown(S);
      } else {
        S->alpha = nu / mu;
      }
    }
  }
}

// u_0 = A s~_0 (pipelined variants).
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_init_c(Op op, Pc pc, Vecs V, DevState* S) {
  if (__ldcg(&S->done)) return;
  const double* __restrict__ st = Pc::on ? V.st[0] : V.s[0];
  PRCG_ROWS(i, op.n) { V.u[0][i] = op.row(i, [&](int j) { return __ldg(st + j); }); }
}

// ---------------------------------------------------------------- HS-CG
// Sweep A of iteration k: x_k, r_k, nu_k = <M^{-1} r_k, r_k>; then beta_k.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_hs_a(Op op, Pc pc, Vecs V, DevState* S,
                                                 double* partials, int qr) {
  if (__ldcg(&S->done)) return;
  const double alpha = __ldcg(&S->alpha);
  double acc[2] = {0.0, 0.0};
  const double* __restrict__ p = V.p[qr];
  double* __restrict__ r = V.r[0];
  const double* __restrict__ s = V.s[0];
  double* __restrict__ x = V.x;
  PRCG_ROWS(i, op.n) {
    x[i] = fma(alpha, __ldg(p + i), x[i]);
    const double rn = fma(-alpha, s[i], r[i]);
    r[i] = rn;
    const double rt = Pc::on ? pc(i) * rn : rn;
    acc[0] += rt * rn;
    acc[1] += rn * rn;
  }
  double tot[2];
  if (grid_sum<2>(acc, partials, S, tot) && threadIdx.x == 0) {
    const int k = S->k + 1;
    const double nu = tot[0];
    if (!record_and_test(S, k, Pc::on ? tot[1] : tot[0])) {
      if (!finite(nu) || !(nu > 0.0)) {
        breakdown(S);
      } else {
        S->beta = nu / S->nu;
        S->nu = nu;
      }
    }
    S->rho = tot[1];
  }
}

// Sweep B of iteration k: p_k = M^{-1} r_k + beta_k p_{k-1}, s_k = A p_k,
// mu_k = <p_k, s_k>; then alpha_k.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_hs_b(Op op, Pc pc, Vecs V, DevState* S,
                                                 double* partials, int qr, int qw) {
  if (__ldcg(&S->done)) return;
  const double beta = __ldcg(&S->beta);
  double acc[1] = {0.0};
  const double* __restrict__ p = V.p[qr];
  const double* __restrict__ r = V.r[0];
  auto pnew = [&](int j) {
    const double rj = __ldg(r + j);
    const double rt = Pc::on ? pc(j) * rj : rj;
    return fma(beta, __ldg(p + j), rt);
  };
  PRCG_ROWS(i, op.n) {
    const double pn = pnew(i);
    const double sn = op.row(i, pnew);
    V.p[qw][i] = pn;
    V.s[0][i] = sn;
    acc[0] += pn * sn;
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, S, tot) && threadIdx.x == 0) {
    const double nu = S->nu, mu = tot[0];
    S->mu = mu;
    if (!finite(mu) || !(mu > 0.0)) {
      breakdown(S);
    } else {
      S->alpha = nu / mu;
    }
  }
}

// ---------------------------------------------------------------- PR-CG / M-CG
// One sweep per iteration k (Algorithm 2): x_k, r_k, r~_k, p_k, s_k = A p_k,
// s~_k = M^{-1} s_k and the four inner products mu, sigma, gamma, nu (and
// <r_k, r_k> when preconditioned), then alpha_k, nu'_{k+1}, beta_{k+1}.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_pr(Op op, Pc pc, Vecs V, DevState* S,
                                               double* partials, int qr, int qw, int meurant) {
  if (__ldcg(&S->done)) return;
  const double alpha = __ldcg(&S->alpha);
  const double beta = __ldcg(&S->beta);
  const double* __restrict__ p = V.p[qr];
  const double* __restrict__ r = V.r[qr];
  const double* __restrict__ rt = Pc::on ? V.rt[qr] : V.r[qr];
  const double* __restrict__ s = V.s[qr];
  double* __restrict__ x = V.x;
  // p_k at column j from the previous iteration's vectors
  auto pnew = [&](int j) {
    const double sj = __ldg(s + j);
    const double rtn = Pc::on ? fma(-alpha, pc(j) * sj, __ldg(rt + j)) : fma(-alpha, sj, __ldg(r + j));
    return fma(beta, __ldg(p + j), rtn);
  };
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  PRCG_ROWS(i, op.n) {
    const double pi = __ldg(p + i);
    const double si = __ldg(s + i);
    x[i] = fma(alpha, pi, x[i]);
    const double rn = fma(-alpha, si, __ldg(r + i));
    const double rtn = Pc::on ? fma(-alpha, pc(i) * si, __ldg(rt + i)) : rn;
    const double pn = fma(beta, pi, rtn);
    const double sn = op.row(i, pnew);
    const double stn = Pc::on ? pc(i) * sn : sn;
    V.r[qw][i] = rn;
    if (Pc::on) V.rt[qw][i] = rtn;
    V.p[qw][i] = pn;
    V.s[qw][i] = sn;
    acc[0] += pn * sn;    // mu_k
    acc[1] += rtn * sn;   // sigma_k
    acc[2] += stn * sn;   // gamma_k
    acc[3] += rtn * rn;   // nu_k
    acc[4] += rn * rn;    // <r_k, r_k>
  }
  double tot[5];
  if (grid_sum<5>(acc, partials, S, tot) && threadIdx.x == 0) {
    const int k = S->k + 1;
    S->mu = tot[0];
    S->sigma = tot[1];
    S->gamma = tot[2];
    S->nu = tot[3];
    S->rho = tot[4];
    if (!record_and_test(S, k, Pc::on ? tot[4] : tot[3])) scalar_step_pr(S, meurant != 0);
  }
}

// ---------------------------------------------------------- pipe-PR-CG / pipe-M
// One sweep per iteration k (Algorithm 3 with the scalars first, Section
// 2.2.1): x_k, r_k, r~_k, w'_k, w~'_k, p_k, s_k, s~_k, then u_k = A s~_k and
// the recomputed w_k = A r~_k in one pass over A, the inner products, and
// alpha_k, nu'_{k+1}, beta_{k+1}.  w~ and u~ are M^{-1} w and M^{-1} u and
// are formed where they are used instead of being stored.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_pipe(Op op, Pc pc, Vecs V, DevState* S,
                                                 double* partials, int qr, int qw, int meurant) {
  if (__ldcg(&S->done)) return;
  const double alpha = __ldcg(&S->alpha);
  const double beta = __ldcg(&S->beta);
  const double* __restrict__ p = V.p[qr];
  const double* __restrict__ r = V.r[qr];
  const double* __restrict__ rt = Pc::on ? V.rt[qr] : V.r[qr];
  const double* __restrict__ s = V.s[qr];
  const double* __restrict__ st = Pc::on ? V.st[qr] : V.s[qr];
  const double* __restrict__ w = V.w[qr];
  const double* __restrict__ u = V.u[qr];
  double* __restrict__ x = V.x;
  // r~_k at column j
  auto rtnew = [&](int j) { return fma(-alpha, __ldg(st + j), __ldg(rt + j)); };
  // s~_k = w~'_k + beta_k s~_{k-1} at column j
  auto stnew = [&](int j) {
    if (Pc::on) {
      const double dj = pc(j);
      return fma(beta, __ldg(st + j), fma(-alpha, dj * __ldg(u + j), dj * __ldg(w + j)));
    }
    return fma(beta, __ldg(st + j), fma(-alpha, __ldg(u + j), __ldg(w + j)));
  };
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  PRCG_ROWS(i, op.n) {
    const double pi = __ldg(p + i);
    const double si = __ldg(s + i);
    const double wi = __ldg(w + i);
    const double ui = __ldg(u + i);
    x[i] = fma(alpha, pi, x[i]);
    const double rn = fma(-alpha, si, __ldg(r + i));
    const double rtn = Pc::on ? rtnew(i) : rn;
    const double wp = fma(-alpha, ui, wi);
    const double pn = fma(beta, pi, rtn);
    const double sn = fma(beta, si, wp);
    const double stn = Pc::on ? stnew(i) : sn;
    double un, wn;
    op.row2(i, stnew, rtnew, un, wn);
    V.r[qw][i] = rn;
    if (Pc::on) {
      V.rt[qw][i] = rtn;
      V.st[qw][i] = stn;
    }
    V.p[qw][i] = pn;
    V.s[qw][i] = sn;
    V.w[qw][i] = wn;
    V.u[qw][i] = un;
    acc[0] += pn * sn;
    acc[1] += rtn * sn;
    acc[2] += stn * sn;
    acc[3] += rtn * rn;
    acc[4] += rn * rn;
  }
  double tot[5];
  if (grid_sum<5>(acc, partials, S, tot) && threadIdx.x == 0) {
    const int k = S->k + 1;
    S->mu = tot[0];
    S->sigma = tot[1];
    S->gamma = tot[2];
    S->nu = tot[3];
    S->rho = tot[4];
    if (!record_and_test(S, k, Pc::on ? tot[4] : tot[3])) scalar_step_pr(S, meurant != 0);
  }
}

// ---------------------------------------------------------------- helpers
// ||b - A x||^2 and ||b||^2 into S->eta and S->nu_pred (after the run).
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_true_res(Op op, Pc pc, Vecs V, DevState* S,
                                                     double* partials) {
  double acc[2] = {0.0, 0.0};
  const double* __restrict__ x = V.x;
  PRCG_ROWS(i, op.n) {
    const double bi = __ldg(V.b + i);
    const double t = bi - op.row(i, [&](int j) { return __ldg(x + j); });
    acc[0] += t * t;
    acc[1] += bi * bi;
  }
  double tot[2];
  if (grid_sum<2>(acc, partials, S, tot) && threadIdx.x == 0) {
    S->eta = tot[0];
    S->nu_pred = tot[1];
  }
}

}  // namespace prcg
