// Sweeps of HS-CG (Algorithm 1), PR-CG / M-CG (Algorithm 2 and its
// Appendix E variant) and pipe-PR-CG / pipe-PR-M-CG (Algorithm 3).
//
// On GB300 an FP64 operation costs more than the bytes it touches (the SMs
// issue 2 FP64 FMAs per clock each), so every sweep performs each
// arithmetic operation of the algorithm exactly once: a vector that a
// matrix-vector product gathers is stored by the sweep that forms it and
// read back by the next one, never recomputed at every column that uses it.
// The dependency structure of each variant then fixes the number of sweeps
// per iteration:
//   HS-CG    3 sweeps, 2 reductions: x,r | p | s = A p
//   PR-CG    2 sweeps, 1 reduction:  x,r,r~,p | s = A p + all inner products
//   pipe-PR  1 sweep,  1 reduction:  u = A s~, w = A r~ of iteration k-1
//            fused with the vector updates and inner products of iteration
//            k (the recurrences of Section 2.2 make the products of k-1 the
//            only thing iteration k's updates need from other rows).
// Each sweep ends, where the variant has a reduction there, with the grid
// reduction of grid_sum; its last CTA forms the next scalars on the device.
#pragma once

#include "prcg_ops.cuh"

namespace prcg {

// CTAs per SM the single-product sweeps ask the register allocator for.
// The constant stencil's product sweeps are bound by memory latency: PR's
// takes two pairs of rows a loop trip so that their loads are in flight
// together, which needs up to 64 registers (4 CTAs of 256 threads); HS's,
// one pair a trip at 6 CTAs (40 registers), below.  0 leaves the allocator
// its own choice (the other operators, and the two-product pipelined
// sweep).
template <class Op>
struct SweepMinBlocks {
  static constexpr int value = 0;
};
template <int DIM>
struct SweepMinBlocks<StencilOp<DIM>> {
  static constexpr int value = 4;
};

// HS-CG's product sweep does one inner product a row (PR-CG's three): it
// gains more from warps than from the two-pair loop trips of PR's sweep.
template <class Op>
struct HsProductMinBlocks {
  static constexpr int value = SweepMinBlocks<Op>::value;
};
template <int DIM>
struct HsProductMinBlocks<StencilOp<DIM>> {
  static constexpr int value = 6;
};

// t - alpha (M^{-1} v)_i: the update of a recurrence for a preconditioned
// vector (r~ of PR-CG, w~' of pipe-PR-CG).  For a Jacobi vector d it forms
// the explicit d_i v_i of the algorithm and one FMA; for a constant d the
// caller passes ad = alpha d, formed once per sweep, and the update is one
// FMA -- the same quantity reassociated, one FP64 instruction less per row
// on the FP64-starved sweeps (the constant d is likewise factored out of the
// inner products <r, r~> and <s, s~>).
template <class Pc>
__device__ __forceinline__ double sub_scaled(const Pc& pc, int i, double alpha, double ad,
                                             double v, double t) {
  if constexpr (std::is_same<Pc, PcScalar>::value)
    return fma(-ad, v, t);
  else
    return fma(-alpha, pc(i) * v, t);
}

// w~'_k = M^{-1} w_{k-1} - alpha M^{-1} u_{k-1} of pipe-PR-CG (Algorithm 3)
// from the row's products u, w and w'_k = w - alpha u.  M^{-1} = diag(d)
// is applied row by row, so d_i w_i - alpha d_i u_i = d_i (w_i - alpha u_i)
// = d_i w'_k: the same quantity reassociated, one multiply instead of the
// two explicit products and an FMA (two FP64 instructions less per row).
template <class Pc>
__device__ __forceinline__ double wt_pred(const Pc& pc, int i, double wp) {
  return pc(i) * wp;
}

// Scale of the block fixed-point copy of the next p, from upper bounds of
// the magnitudes it is formed from (thread 0 of a last CTA, after the scalar
// step).  PR-CG / M-CG: p_{k+1} = r~_{k+1} + beta_{k+1} p_k with
// r~_{k+1} = r~_k - alpha_k d s_k, so |p_{k+1}| <= max|r~_k| +
// |alpha_k d| max|s_k| + |beta_{k+1}| max|p_k|.  HS-CG: p_k = d r_k +
// beta_k p_{k-1}, so |p_k| <= d max|r_k| + |beta_k| max|p_{k-1}|.  A factor
// 1 + 2^-40 covers the roundings of the bound and of the updates; the
// trackers are then cleared for the next iteration.
template <class Pc>
__device__ __forceinline__ void set_fixed_scale(DevState* S, const Pc& pc, double bound) {
  const int sc = fixed_scale(bound * (1.0 + 0x1p-40));
  S->pf_on = (S->pf_allow && !S->done && sc != kNoScale) ? 1 : 0;
  S->pf_scale = sc;
  S->pf_bad = 0;
}

template <class Pc>
__device__ __forceinline__ void next_fixed_scale_pr(DevState* S, const Pc& pc) {
  const double d = Pc::on ? pc(0) : 1.0;
  const double B = amax_bound(S->amax_r) + fabs(S->alpha * d) * amax_bound(S->amax_s) +
                   fabs(S->beta) * amax_bound(S->amax_p);
  set_fixed_scale(S, pc, B);
  S->amax_r = 0u;
  S->amax_p = 0u;
  S->amax_s = 0u;
}

template <class Pc>
__device__ __forceinline__ void next_fixed_scale_hs(DevState* S, const Pc& pc) {
  const double d = Pc::on ? pc(0) : 1.0;
  const double B = d * amax_bound(S->amax_r) + fabs(S->beta) * amax_bound(S->amax_p);
  set_fixed_scale(S, pc, B);
  S->amax_r = 0u;
  S->amax_p = 0u;
}

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
  constexpr bool kFx = HasFixedRow<Op>::value;
  double acc[3] = {0.0, 0.0, 0.0};
  unsigned mr = 0u;
  const double* __restrict__ x = V.x;
  PRCG_ROWS(i, op.n) {
    const double ax = op.row(i, [&](int j) { return __ldg(x + j); });
    const double bi = __ldg(V.b + i);
    const double r = bi - ax;
    const double rt = Pc::on ? pc(i) * r : r;
    V.r[0][i] = r;
    if (Pc::on) V.rt[0][i] = rt;
    V.p[0][i] = rt;
    if (kFx) mr = max(mr, mag_hi(rt));
    acc[0] += rt * r;
    acc[1] += r * r;
    acc[2] += bi * bi;
  }
  if (kFx) {   // max |r~_0| = max |p_0|, for the scale of the first fixed-point p
    cta_atomic_max(mr, &S->amax_r);
    cta_atomic_max(mr, &S->amax_p);
  }
  double tot[3];
  if (grid_sum<3>(acc, partials, S, tot) && threadIdx.x == 0) {
    S->nu = tot[0];
    S->rho = tot[1];
    S->bnorm2 = tot[2];
    S->k = 0;
    trace(S, 0, TR_NU, tot[0]);
    trace(S, 0, TR_RHO, tot[1]);
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

// s_0 = A p_0, s~_0 = M^{-1} s_0 (stored for the pipelined variants, whose
// s~ is a recurrence); mu_0, sigma_0, gamma_0; then alpha_0 (and nu'_1,
// beta_1 for the predict-and-recompute variants).
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_init_b(Op op, Pc pc, Vecs V, DevState* S,
                                                   double* partials, int variant) {
  if (__ldcg(&S->done)) return;
  const bool pipe = variant == V_PIPE || variant == V_PIPE_M || variant == V_GV ||
                    variant == V_PIPE_NR;
  const bool keep_w = variant == V_CGCG || variant == V_GV || variant == V_PIPE_NR;
  constexpr bool kFx = HasFixedRow<Op>::value;
  double acc[3] = {0.0, 0.0, 0.0};
  unsigned ms = 0u;
  const double* __restrict__ p = V.p[0];
  PRCG_ROWS(i, op.n) {
    const double s = op.row(i, [&](int j) { return __ldg(p + j); });
    const double st = Pc::on ? pc(i) * s : s;
    if (kFx) ms = max(ms, mag_hi(s));
    V.s[0][i] = s;
    if (Pc::on && pipe) V.st[0][i] = st;
    if (keep_w) V.w[0][i] = s;   // w_0 = A r~_0 is the same product (p_0 = r~_0)
    if (variant == V_GV) V.u[0][i] = 0.0;   // multiplied by beta_0 = 0 in the first sweep
    if (variant == V_PIPE_NR && Pc::on) V.u[0][i] = st;   // w~_0 = M^{-1} w_0
    const double pi = __ldg(p + i);
    const double rt = Pc::on ? __ldg(V.rt[0] + i) : __ldg(V.r[0] + i);
    acc[0] += pi * s;
    acc[1] += rt * s;
    acc[2] += st * s;
  }
  if (kFx) cta_atomic_max(ms, &S->amax_s);
  double tot[3];
  if (grid_sum<3>(acc, partials, S, tot) && threadIdx.x == 0) {
    S->mu = tot[0];
    S->sigma = tot[1];
    S->gamma = tot[2];
    trace(S, 0, TR_MU, tot[0]);
    trace(S, 0, TR_SIGMA, tot[1]);
    trace(S, 0, TR_GAMMA, tot[2]);
    if (variant == V_PR || variant == V_PIPE || variant == V_M || variant == V_PIPE_M ||
        variant == V_PR_NR || variant == V_PIPE_NR) {
      scalar_step_pr(S, variant == V_M || variant == V_PIPE_M);
      if (kFx && (variant == V_PR || variant == V_M || variant == V_PR_NR))
        next_fixed_scale_pr(S, pc);
    } else {
      const double nu = S->nu, mu = tot[0];
      if (!finite(nu) || !finite(mu) || !(mu > 0.0) || nu < 0.0) {
        breakdown(S);
      } else {
        S->alpha = nu / mu;
        trace(S, 1, TR_ALPHA, S->alpha);
        // CG-CG / GV-CG: the first sweep "updates" p_0, s_0 (, s~_0, u_0)
        // with beta_0 = 0, which leaves the initial vectors as they are
        S->beta = 0.0;
      }
    }
  }
}

// ---------------------------------------------------------------- HS-CG
// Sweep A of iteration k: x_k, r_k, nu_k = <M^{-1} r_k, r_k>, <r_k, r_k>;
// then the stopping test and beta_k = nu_k / nu_{k-1}.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_hs_a(Op op, Pc pc, Vecs V, DevState* S,
                                                 double* partials) {
  if (__ldcg(&S->done)) return;
  const double alpha = __ldcg(&S->alpha);
  double acc[2] = {0.0, 0.0};
  const double* __restrict__ p = V.p[0];
  double* __restrict__ r = V.r[0];
  const double* __restrict__ s = V.s[0];
  double* __restrict__ x = V.x;
  constexpr bool kNuDot = Pc::on && !std::is_same<Pc, PcScalar>::value;
  constexpr bool kFx = HasFixedRow<Op>::value;
  unsigned mr = 0u;
  auto update = [&](double pi, double si, double& xi, double& ri, double di) {
    xi = fma(alpha, pi, xi);
    const double rn = fma(-alpha, si, ri);
    ri = rn;
    if (kFx) mr = max(mr, mag_hi(rn));
    acc[1] = fma(rn, rn, acc[1]);
    if (kNuDot) acc[0] = fma(di * rn, rn, acc[0]);
  };
  // two rows per thread with 16-byte accesses (as in k_pr_a)
  const int n = op.n, npair = n >> 1;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < npair; j += gridDim.x * blockDim.x) {
    const int i = 2 * j;
    const double2 p2 = __ldg(reinterpret_cast<const double2*>(p + i));
    const double2 s2 = __ldg(reinterpret_cast<const double2*>(s + i));
    double2 x2 = *reinterpret_cast<const double2*>(x + i);
    double2 r2 = *reinterpret_cast<const double2*>(r + i);
    const double2 d2 = kNuDot ? pc_pair(pc, i) : make_double2(1.0, 1.0);
    update(p2.x, s2.x, x2.x, r2.x, d2.x);
    update(p2.y, s2.y, x2.y, r2.y, d2.y);
    *reinterpret_cast<double2*>(x + i) = x2;
    *reinterpret_cast<double2*>(r + i) = r2;
  }
  if ((n & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const int i = n - 1;
    double xi = x[i], ri = r[i];
    update(__ldg(p + i), __ldg(s + i), xi, ri, kNuDot ? pc(i) : 1.0);
    x[i] = xi;
    r[i] = ri;
  }
  if (kFx) cta_atomic_max(mr, &S->amax_r);
  double tot[2];
  if (grid_sum<2>(acc, partials, S, tot) && threadIdx.x == 0) {
    const int k = S->k + 1;
    // nu_k: <r, r> unpreconditioned; d <r, r> for a constant Jacobi d
    double nu = tot[0];
    if (!Pc::on) nu = tot[1];
    if (std::is_same<Pc, PcScalar>::value) nu = pc(0) * tot[1];
    S->rho = tot[1];
    trace(S, k, TR_NU, nu);
    trace(S, k, TR_RHO, tot[1]);
    if (!record_and_test(S, k, tot[1])) {
      if (!finite(nu) || !(nu > 0.0)) {
        breakdown(S);
      } else {
        S->beta = nu / S->nu;
        S->nu = nu;
        trace(S, k, TR_BETA, S->beta);
        if (kFx) next_fixed_scale_hs(S, pc);
      }
    }
  }
}

// Sweep B of iteration k: p_k = M^{-1} r_k + beta_k p_{k-1} (row-local).
// For a constant stencil it also stores the block fixed-point copy of p_k
// (scale chosen by sweep A) and tracks max |p_k|.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_hs_b(Op op, Pc pc, Vecs V, DevState* S) {
  if (__ldcg(&S->done)) return;
  const double beta = __ldcg(&S->beta);
  double* __restrict__ p = V.p[0];
  const double* __restrict__ r = V.r[0];
  constexpr bool kFx = HasFixedRow<Op>::value;
  const bool fx = kFx && __ldcg(&S->pf_on);
  const int sc = kFx ? __ldcg(&S->pf_scale) : 0;
  unsigned mp = 0u;
  bool bad = false;
  // two rows per thread with 16-byte accesses (as in k_pr_a)
  const int n = op.n, npair = n >> 1;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < npair; j += gridDim.x * blockDim.x) {
    const int i = 2 * j;
    const double2 r2 = __ldg(reinterpret_cast<const double2*>(r + i));
    const double2 d2 = Pc::on ? pc_pair(pc, i) : make_double2(1.0, 1.0);
    double2 p2 = *reinterpret_cast<const double2*>(p + i);
    p2.x = fma(beta, p2.x, Pc::on ? d2.x * r2.x : r2.x);
    p2.y = fma(beta, p2.y, Pc::on ? d2.y * r2.y : r2.y);
    *reinterpret_cast<double2*>(p + i) = p2;
    if (kFx) {
      mp = max(mp, max(mag_hi(p2.x), mag_hi(p2.y)));
      if (fx) {
        longlong2 q;
        q.x = to_fixed(p2.x, sc, bad);
        q.y = to_fixed(p2.y, sc, bad);
        *reinterpret_cast<longlong2*>(V.pf + i) = q;
      }
    }
  }
  if ((n & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const int i = n - 1;
    const double ri = __ldg(r + i);
    const double pn = fma(beta, p[i], Pc::on ? pc(i) * ri : ri);
    p[i] = pn;
    if (kFx) {
      mp = max(mp, mag_hi(pn));
      if (fx) V.pf[i] = to_fixed(pn, sc, bad);
    }
  }
  if (kFx) {
    if (fx && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&S->pf_bad, 1);
    cta_atomic_max(mp, &S->amax_p);
  }
}

// Sweep C of iteration k: s_k = A p_k, mu_k = <p_k, s_k>; then alpha_k.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock, HsProductMinBlocks<Op>::value)
    k_hs_c(Op op, Pc pc, Vecs V, DevState* S, double* partials) {
  if (__ldcg(&S->done)) return;
  double acc[1] = {0.0};
  const double* __restrict__ p = V.p[0];
  bool fixed_done = false;
  if constexpr (HasFixedRow<Op>::value) {
    if (__ldcg(&S->pf_on) && !__ldcg(&S->pf_bad)) {
      // the neighbour sums from the block fixed-point copy of p_k
      const int sc = __ldcg(&S->pf_scale);
      const long long* __restrict__ P = V.pf;
      // kInt: the whole row in integers (an integer diagonal), a separate
      // loop so that no predicated FMA is issued for it
      auto sweep = [&](auto kInt) {
        constexpr bool KI = decltype(kInt)::value;
        if ((op.nx & 1) == 0) {
          // pairs of rows of one x-line, 16-byte accesses (n is even)
          for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < (op.n >> 1);
               j += gridDim.x * blockDim.x) {
            const int i = 2 * j;
            const double2 p2 = __ldg(reinterpret_cast<const double2*>(p + i));
            const double2 s2 = op.template rows2_fixed<KI>(i, p2, P, sc);
            *reinterpret_cast<double2*>(V.s[0] + i) = s2;
            acc[0] = fma(p2.x, s2.x, acc[0]);
            acc[0] = fma(p2.y, s2.y, acc[0]);
          }
        } else {
          PRCG_ROWS(i, op.n) {
            const double pi = __ldg(p + i);
            const double sn = op.template row_fixed<KI>(i, pi, P, sc);
            V.s[0][i] = sn;
            acc[0] = fma(pi, sn, acc[0]);
          }
        }
      };
      if (op.cint)
        sweep(std::true_type{});
      else
        sweep(std::false_type{});
      fixed_done = true;
    }
  }
  bool paired = false;
  if constexpr (HasRows2<Op>::value) {
    if (!fixed_done && op.pairs_ok()) {
      // two rows of one grid line per thread, 16-byte loads (n is even)
      auto g = [&](int j) { return __ldg(p + j); };
      auto g2 = [&](int j) { return __ldg(reinterpret_cast<const double2*>(p + j)); };
      for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < (op.n >> 1);
           j += gridDim.x * blockDim.x) {
        const int i = 2 * j;
        const double2 s2 = op.rows2(i, g, g2);
        *reinterpret_cast<double2*>(V.s[0] + i) = s2;
        const double2 p2 = g2(i);
        acc[0] = fma(p2.x, s2.x, acc[0]);
        acc[0] = fma(p2.y, s2.y, acc[0]);
      }
      paired = true;
    }
  }
  if (!fixed_done && !paired) {
    PRCG_ROWS(i, op.n) {
      const double sn = op.row(i, [&](int j) { return __ldg(p + j); });
      V.s[0][i] = sn;
      acc[0] = fma(__ldg(p + i), sn, acc[0]);
    }
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, S, tot) && threadIdx.x == 0) {
    if (fixed_done) ++S->pf_sweeps;
    const double mu = tot[0];
    S->mu = mu;
    trace(S, S->k, TR_MU, mu);
    if (!finite(mu) || !(mu > 0.0)) {
      breakdown(S);
    } else {
      S->alpha = S->nu / mu;
      trace(S, S->k + 1, TR_ALPHA, S->alpha);
    }
  }
}

// ---------------------------------------------------------------- PR-CG / M-CG
// Sweep A of iteration k (Algorithm 2, the scalars formed up front):
// x_k, r_k, r~_k = r~_{k-1} - alpha s~_{k-1} (s~ = M^{-1} s, formed here),
// p_k = r~_k + beta_k p_{k-1}; partial sums of nu_k = <r~_k, r_k> and
// <r_k, r_k> go to partials_a and are added by sweep B's reduction.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_pr_a(Op op, Pc pc, Vecs V, DevState* S,
                                                 double* partials_a) {
  if (__ldcg(&S->done)) return;
  const double alpha = __ldcg(&S->alpha);
  const double beta = __ldcg(&S->beta);
  const double ad = std::is_same<Pc, PcScalar>::value ? alpha * pc(0) : 0.0;
  double* __restrict__ x = V.x;
  double* __restrict__ r = V.r[0];
  double* __restrict__ rt = V.rt[0];
  double* __restrict__ p = V.p[0];
  const double* __restrict__ s = V.s[0];
  double acc[2] = {0.0, 0.0};
  // constant stencil: max |r~_k|, max |p_k| and the block fixed-point copy
  // of p_k (scale chosen by the previous reduction) for sweep B
  constexpr bool kFx = HasFixedRow<Op>::value;
  const bool fx = kFx && __ldcg(&S->pf_on);
  const int sc = kFx ? __ldcg(&S->pf_scale) : 0;
  unsigned mr = 0u, mp = 0u;
  bool bad = false;
  // the update of one row from its old values; returns rtn and writes x, r, p
  auto update = [&](double si, double pi, double& xi, double& ri, double& rti, double di) {
    xi = fma(alpha, pi, xi);
    const double rn = fma(-alpha, si, ri);
    ri = rn;
    double rtn = rn;
    if (Pc::on) {
      rtn = std::is_same<Pc, PcScalar>::value ? fma(-ad, si, rti) : fma(-alpha, di * si, rti);
      rti = rtn;
      acc[0] = fma(rtn, rn, acc[0]);
    }
    acc[1] = fma(rn, rn, acc[1]);
    const double pn = fma(beta, pi, rtn);   // p_k
    if (kFx) {
      mr = max(mr, mag_hi(rtn));
      mp = max(mp, mag_hi(pn));
    }
    return pn;
  };
  // two rows per thread: 16-byte loads and stores halve the memory requests
  // of this streaming sweep (vectors start on 256-byte boundaries)
  const int n = op.n, npair = n >> 1;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < npair; j += gridDim.x * blockDim.x) {
    const int i = 2 * j;
    const double2 s2 = __ldg(reinterpret_cast<const double2*>(s + i));
    const double2 p2 = *reinterpret_cast<const double2*>(p + i);
    double2 x2 = *reinterpret_cast<const double2*>(x + i);
    double2 r2 = *reinterpret_cast<const double2*>(r + i);
    double2 rt2 = Pc::on ? *reinterpret_cast<const double2*>(rt + i) : make_double2(0.0, 0.0);
    const double2 d2 = pc_pair(pc, i);
    double2 pn;
    pn.x = update(s2.x, p2.x, x2.x, r2.x, rt2.x, d2.x);
    pn.y = update(s2.y, p2.y, x2.y, r2.y, rt2.y, d2.y);
    *reinterpret_cast<double2*>(x + i) = x2;
    *reinterpret_cast<double2*>(r + i) = r2;
    if (Pc::on) *reinterpret_cast<double2*>(rt + i) = rt2;
    *reinterpret_cast<double2*>(p + i) = pn;
    if (fx) {
      longlong2 q;
      q.x = to_fixed(pn.x, sc, bad);
      q.y = to_fixed(pn.y, sc, bad);
      *reinterpret_cast<longlong2*>(V.pf + i) = q;
    }
  }
  if ((n & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const int i = n - 1;
    double xi = x[i], ri = r[i], rti = Pc::on ? rt[i] : 0.0;
    const double pn = update(__ldg(s + i), p[i], xi, ri, rti, Pc::on ? pc(i) : 1.0);
    p[i] = pn;
    if (fx) V.pf[i] = to_fixed(pn, sc, bad);
    x[i] = xi;
    r[i] = ri;
    if (Pc::on) rt[i] = rti;
  }
  if (kFx) {
    if (fx && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&S->pf_bad, 1);
    cta_atomic_max(mr, &S->amax_r);
    cta_atomic_max(mp, &S->amax_p);
  }
  __shared__ double sm[2 * 32];
  block_sum<2>(acc, sm);
  if (threadIdx.x == 0) {
    partials_a[blockIdx.x * 2 + 0] = acc[0];
    partials_a[blockIdx.x * 2 + 1] = acc[1];
  }
}

// Sweep B of iteration k: s_k = A p_k and mu_k, sigma_k = <r~_k, s_k>,
// gamma_k = <M^{-1} s_k, s_k>; the reduction adds sweep A's nu_k and
// <r_k, r_k>, tests for convergence and forms alpha_k, nu'_{k+1} (Eq. 2.3
// or Meurant's form), beta_{k+1}.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock, SweepMinBlocks<Op>::value)
    k_pr_b(Op op, Pc pc, Vecs V, DevState* S, double* partials, const double* partials_a,
           int grid_a, int meurant) {
  if (__ldcg(&S->done)) return;
  const double* __restrict__ p = V.p[0];
  const double* __restrict__ rt = Pc::on ? V.rt[0] : V.r[0];
  double acc[3] = {0.0, 0.0, 0.0};
  constexpr bool kFx = HasFixedRow<Op>::value;
  unsigned ms = 0u;
  auto sums = [&](int i, double pi, double sn) {
    V.s[0][i] = sn;
    acc[0] = fma(pi, sn, acc[0]);
    acc[1] = fma(__ldg(rt + i), sn, acc[1]);
    if (std::is_same<Pc, PcVec>::value)
      acc[2] = fma(pc(i) * sn, sn, acc[2]);
    else
      acc[2] = fma(sn, sn, acc[2]);
    if (kFx) ms = max(ms, mag_hi(sn));
  };
  bool fixed_done = false;
  if constexpr (kFx) {
    if (__ldcg(&S->pf_on) && !__ldcg(&S->pf_bad)) {
      // the neighbour sums from the block fixed-point copy of p_k
      const int sc = __ldcg(&S->pf_scale);
      const long long* __restrict__ P = V.pf;
      static_assert(!std::is_same<Pc, PcVec>::value, "constant stencils have a scalar d");
      // kInt: the whole row in integers (an integer diagonal), a separate
      // loop so that no predicated FMA is issued for it
      auto sweep = [&](auto kInt) {
        constexpr bool KI = decltype(kInt)::value;
        if ((op.nx & 1) == 0) {
          // pairs of rows of one x-line, 16-byte accesses (n is even); two
          // pairs a loop trip, their loads issued together
          double* __restrict__ sv = V.s[0];
          const int np = op.n >> 1, str = gridDim.x * blockDim.x;
          auto pair_sums = [&](double2 p2, double2 r2, double2 s2) {
            acc[0] = fma(p2.x, s2.x, acc[0]);
            acc[1] = fma(r2.x, s2.x, acc[1]);
            acc[2] = fma(s2.x, s2.x, acc[2]);
            acc[0] = fma(p2.y, s2.y, acc[0]);
            acc[1] = fma(r2.y, s2.y, acc[1]);
            acc[2] = fma(s2.y, s2.y, acc[2]);
            ms = max(ms, max(mag_hi(s2.x), mag_hi(s2.y)));
          };
          for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < np; j += 2 * str) {
            const bool hb = j + str < np;
            const int ia = 2 * j, ib = hb ? 2 * (j + str) : ia;
            const double2 pa = __ldg(reinterpret_cast<const double2*>(p + ia));
            const double2 pb = __ldg(reinterpret_cast<const double2*>(p + ib));
            const double2 ra = __ldg(reinterpret_cast<const double2*>(rt + ia));
            const double2 rb = __ldg(reinterpret_cast<const double2*>(rt + ib));
            const double2 sa = op.template rows2_fixed<KI>(ia, pa, P, sc);
            const double2 sb = op.template rows2_fixed<KI>(ib, pb, P, sc);
            *reinterpret_cast<double2*>(sv + ia) = sa;
            pair_sums(pa, ra, sa);
            if (hb) {
              *reinterpret_cast<double2*>(sv + ib) = sb;
              pair_sums(pb, rb, sb);
            }
          }
        } else {
          PRCG_ROWS(i, op.n) {
            const double pi = __ldg(p + i);
            sums(i, pi, op.template row_fixed<KI>(i, pi, P, sc));
          }
        }
      };
      if (op.cint)
        sweep(std::true_type{});
      else
        sweep(std::false_type{});
      fixed_done = true;
    }
  }
  bool paired = false;
  if constexpr (HasRows2<Op>::value) {
    if (!fixed_done && op.pairs_ok()) {
      // two rows of one grid line per thread, 16-byte loads (n is even)
      auto g = [&](int j) { return __ldg(p + j); };
      auto g2 = [&](int j) { return __ldg(reinterpret_cast<const double2*>(p + j)); };
      for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < (op.n >> 1);
           j += gridDim.x * blockDim.x) {
        const int i = 2 * j;
        const double2 s2 = op.rows2(i, g, g2);
        const double2 p2 = g2(i);
        sums(i, p2.x, s2.x);
        sums(i + 1, p2.y, s2.y);
      }
      paired = true;
    }
  }
  if (!fixed_done && !paired) {
    PRCG_ROWS(i, op.n) {
      const double sn = op.row(i, [&](int j) { return __ldg(p + j); });
      sums(i, __ldg(p + i), sn);
    }
  }
  if (kFx) cta_atomic_max(ms, &S->amax_s);
  double tot[3];
  if (!grid_sum<3>(acc, partials, S, tot)) return;
  if (threadIdx.x == 0 && fixed_done) ++S->pf_sweeps;
  // last CTA: add sweep A's partial sums (fixed order)
  double a2[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < grid_a; b += blockDim.x) {
    a2[0] += __ldcg(&partials_a[b * 2 + 0]);
    a2[1] += __ldcg(&partials_a[b * 2 + 1]);
  }
  __shared__ double sm2[2 * 32];
  block_sum<2>(a2, sm2, (threadIdx.x & ~31) < grid_a);
  if (threadIdx.x == 0) {
    double nu = a2[0], rho = a2[1];
    if (!Pc::on) nu = rho;
    const int k = S->k + 1;
    S->mu = tot[0];
    S->sigma = tot[1];
    S->gamma = std::is_same<Pc, PcScalar>::value ? pc(0) * tot[2] : tot[2];
    S->nu = nu;
    S->rho = rho;
    trace_pr_sums(S, k);
    if (!record_and_test(S, k, rho)) {
      scalar_step_pr(S, meurant != 0);
      if (kFx) next_fixed_scale_pr(S, pc);
    }
  }
}

// ---------------------------------------------------------- pipe-PR-CG / pipe-M
// Scales of the fixed-point copies of r~_{k+1} and s~_{k+1} (thread 0 of the
// last CTA of sweep k, after the scalar step; q = the buffer sweep k + 1
// writes).  With M_r, M_s the maxima of |r~_k|, |s~_k| and ||A||_inf the
// stencil's largest row sum of magnitudes: r~_{k+1} = r~_k - alpha_k s~_k
// gives |r~_{k+1}| <= M_r + |alpha_k| M_s, and s~_{k+1} = d (w_k - alpha_k
// u_k) + beta_{k+1} s~_k with w_k = A r~_k, u_k = A s~_k gives |s~_{k+1}| <=
// d ||A||_inf (M_r + |alpha_k| M_s) + |beta_{k+1}| M_s (d = 1 without a
// preconditioner, where r~ = r and s~ = s).  The factor 1 + 2^-40 covers
// the roundings of the bounds and of the updates; a value outside its
// window still only sets pq_bad (the next sweep then uses per-row sums).
template <class Pc>
__device__ __forceinline__ void next_pipe_scales(DevState* S, const Pc& pc, double anorm, int q) {
  const double d = Pc::on ? pc(0) : 1.0;
  const double Ms = amax_bound(S->amax_s);
  const double Br = amax_bound(S->amax_r) + fabs(S->alpha) * Ms;
  const double Bs = d * anorm * Br + fabs(S->beta) * Ms;
  const int sr = fixed_scale(Br * (1.0 + 0x1p-40));
  const int ss = fixed_scale(Bs * (1.0 + 0x1p-40));
  S->pq_on[q] = (S->pf_allow && !S->done && sr != kNoScale && ss != kNoScale) ? 1 : 0;
  S->pq_scale_r[q] = sr;
  S->pq_scale_s[q] = ss;
  S->pq_bad[q] = 0;
  S->amax_r = 0u;
  S->amax_s = 0u;
}

// One sweep per iteration k >= 1.  For row i it first forms
//   u_{k-1} = A s~_{k-1},  w_{k-1} = A r~_{k-1}      (the recomputed w)
// from the stored s~_{k-1}, r~_{k-1} (buffer qr), then Algorithm 3's updates
//   x_k, r_k, r~_k, w'_k = w_{k-1} - alpha u_{k-1},
//   w~'_k = M^{-1} w_{k-1} - alpha M^{-1} u_{k-1}, p_k, s_k = w'_k + beta s_{k-1},
//   s~_k = w~'_k + beta s~_{k-1}
// (r~_k, s~_k to buffer qw) and the inner products mu, sigma, gamma, nu of
// iteration k; u and w never leave registers.
//
// Constant stencil: the previous sweep also stored block fixed-point copies
// of r~ and s~ (one scale per vector, prcg_isum.cuh) beside the FP64
// vectors, and both products add the neighbours from them with integer
// adds -- with an integer diagonal the whole row (row_fixed<true>), no FP64
// instruction.  Rows go in pairs of one x-line with 16-byte accesses where
// nx is even.  The first two sweeps, and a sweep whose copy had a value
// outside its window, use the per-row exact sums instead.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_pipe(Op op, Pc pc, Vecs V, DevState* S,
                                                 double* partials, int qr, int qw, int meurant) {
  if (__ldcg(&S->done)) return;
  constexpr bool kFx = HasFixedRow<Op>::value;
  const double alpha = __ldcg(&S->alpha);
  const double beta = __ldcg(&S->beta);
  const double* __restrict__ rt_o = Pc::on ? V.rt[qr] : V.r[qr];
  const double* __restrict__ st_o = Pc::on ? V.st[qr] : V.s[qr];
  const double* __restrict__ r_o = V.r[qr];
  const double* __restrict__ s_o = V.s[qr];
  double* __restrict__ x = V.x;
  double* __restrict__ p = V.p[0];
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  // fixed-point copies: read from buffer qr, written to buffer qw
  const bool rd_fx = kFx && __ldcg(&S->pq_on[qr]) && !__ldcg(&S->pq_bad[qr]);
  const bool wr_fx = kFx && __ldcg(&S->pq_on[qw]);
  const int sr_rd = kFx ? __ldcg(&S->pq_scale_r[qr]) : 0;
  const int ss_rd = kFx ? __ldcg(&S->pq_scale_s[qr]) : 0;
  const int sr_wr = kFx ? __ldcg(&S->pq_scale_r[qw]) : 0;
  const int ss_wr = kFx ? __ldcg(&S->pq_scale_s[qw]) : 0;
  const long long* __restrict__ rf_rd = V.rtf[qr];
  const long long* __restrict__ sf_rd = V.stf[qr];
  unsigned mr = 0u, ms = 0u;
  bool bad = false;
  // Algorithm 3's updates of row i from its old values and the two products
  auto step = [&](int i, double u, double w, double si, double ri, double rti, double sti,
                  double& xi, double& pi, double& rn, double& sn, double& rtn, double& stn) {
    xi = fma(alpha, pi, xi);
    rn = fma(-alpha, si, ri);
    const double wp = fma(-alpha, u, w);
    sn = fma(beta, si, wp);
    if (Pc::on) {
      rtn = fma(-alpha, sti, rti);
      stn = fma(beta, sti, wt_pred(pc, i, wp));
    } else {
      rtn = rn;
      stn = sn;
    }
    pi = fma(beta, pi, rtn);
    acc[0] = fma(pi, sn, acc[0]);
    acc[1] = fma(rtn, sn, acc[1]);
    acc[2] = fma(stn, sn, acc[2]);
    if (Pc::on) acc[3] = fma(rtn, rn, acc[3]);   // unpreconditioned: nu_k = rho_k
    acc[4] = fma(rn, rn, acc[4]);
    if (kFx) {
      mr = max(mr, mag_hi(rtn));
      ms = max(ms, mag_hi(stn));
    }
  };
  bool done_rows = false;
  if constexpr (kFx) {
    // kRd: the products from the copies; kInt: with an integer diagonal
    // (separate loops, so that no predicated FP64 instruction issues)
    auto sweep = [&](auto kRd, auto kInt) {
      constexpr bool RD = decltype(kRd)::value, KI = decltype(kInt)::value;
      if (op.pairs_ok()) {
        auto ld2 = [](const double* q, int j) {
          return __ldg(reinterpret_cast<const double2*>(q + j));
        };
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < (op.n >> 1);
             j += gridDim.x * blockDim.x) {
          const int i = 2 * j;
          const double2 rt2 = ld2(rt_o, i), st2 = ld2(st_o, i);
          double2 u2, w2;
          if constexpr (RD) {
            u2 = op.template rows2_fixed<KI>(i, st2, sf_rd, ss_rd);
            w2 = op.template rows2_fixed<KI>(i, rt2, rf_rd, sr_rd);
          } else {
            u2 = op.rows2(i, [&](int c) { return __ldg(st_o + c); },
                          [&](int c) { return ld2(st_o, c); });
            w2 = op.rows2(i, [&](int c) { return __ldg(rt_o + c); },
                          [&](int c) { return ld2(rt_o, c); });
          }
          const double2 s2 = ld2(s_o, i), r2 = ld2(r_o, i);
          double2 x2 = *reinterpret_cast<const double2*>(x + i);
          double2 p2 = *reinterpret_cast<const double2*>(p + i);
          double2 rn, sn, rtn, stn;
          step(i, u2.x, w2.x, s2.x, r2.x, rt2.x, st2.x, x2.x, p2.x, rn.x, sn.x, rtn.x, stn.x);
          step(i + 1, u2.y, w2.y, s2.y, r2.y, rt2.y, st2.y, x2.y, p2.y, rn.y, sn.y, rtn.y,
               stn.y);
          *reinterpret_cast<double2*>(x + i) = x2;
          *reinterpret_cast<double2*>(p + i) = p2;
          *reinterpret_cast<double2*>(V.r[qw] + i) = rn;
          *reinterpret_cast<double2*>(V.s[qw] + i) = sn;
          if (Pc::on) {
            *reinterpret_cast<double2*>(V.rt[qw] + i) = rtn;
            *reinterpret_cast<double2*>(V.st[qw] + i) = stn;
          }
          if (wr_fx) {
            longlong2 fr, fs;
            fr.x = to_fixed(rtn.x, sr_wr, bad);
            fr.y = to_fixed(rtn.y, sr_wr, bad);
            fs.x = to_fixed(stn.x, ss_wr, bad);
            fs.y = to_fixed(stn.y, ss_wr, bad);
            *reinterpret_cast<longlong2*>(V.rtf[qw] + i) = fr;
            *reinterpret_cast<longlong2*>(V.stf[qw] + i) = fs;
          }
        }
      } else {
        PRCG_ROWS(i, op.n) {
          const double rti = __ldg(rt_o + i), sti = __ldg(st_o + i);
          double u, w;
          if constexpr (RD) {
            u = op.template row_fixed<KI>(i, sti, sf_rd, ss_rd);
            w = op.template row_fixed<KI>(i, rti, rf_rd, sr_rd);
          } else {
            op.row2(i, [&](int j) { return __ldg(st_o + j); },
                    [&](int j) { return __ldg(rt_o + j); }, u, w);
          }
          double xi = x[i], pi = p[i], rn, sn, rtn, stn;
          step(i, u, w, __ldg(s_o + i), __ldg(r_o + i), rti, sti, xi, pi, rn, sn, rtn, stn);
          x[i] = xi;
          p[i] = pi;
          V.r[qw][i] = rn;
          V.s[qw][i] = sn;
          if (Pc::on) {
            V.rt[qw][i] = rtn;
            V.st[qw][i] = stn;
          }
          if (wr_fx) {
            V.rtf[qw][i] = to_fixed(rtn, sr_wr, bad);
            V.stf[qw][i] = to_fixed(stn, ss_wr, bad);
          }
        }
      }
    };
    if (!rd_fx)
      sweep(std::false_type{}, std::false_type{});
    else if (op.cint)
      sweep(std::true_type{}, std::true_type{});
    else
      sweep(std::true_type{}, std::false_type{});
    if (wr_fx && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
      atomicOr(&S->pq_bad[qw], 1);
    cta_atomic_max(mr, &S->amax_r);
    cta_atomic_max(ms, &S->amax_s);
    done_rows = true;
  }
  if (!done_rows) {
    PRCG_ROWS(i, op.n) {
      double u, w;
      op.row2(i, [&](int j) { return __ldg(st_o + j); }, [&](int j) { return __ldg(rt_o + j); },
              u, w);
      double xi = x[i], pi = p[i], rn, sn, rtn, stn;
      step(i, u, w, __ldg(s_o + i), __ldg(r_o + i), __ldg(rt_o + i), __ldg(st_o + i), xi, pi, rn,
           sn, rtn, stn);
      x[i] = xi;
      p[i] = pi;
      V.r[qw][i] = rn;
      V.s[qw][i] = sn;
      if (Pc::on) {
        V.rt[qw][i] = rtn;
        V.st[qw][i] = stn;
      }
    }
  }
  double tot[5];
  if (grid_sum<5>(acc, partials, S, tot) && threadIdx.x == 0) {
    const int k = S->k + 1;
    S->mu = tot[0];
    S->sigma = tot[1];
    S->gamma = tot[2];
    S->nu = Pc::on ? tot[3] : tot[4];
    S->rho = tot[4];
    if (kFx && rd_fx) ++S->pf_sweeps;
    trace_pr_sums(S, k);
    if (!record_and_test(S, k, tot[4])) {
      scalar_step_pr(S, meurant != 0);
      if constexpr (kFx) next_pipe_scales(S, pc, op.anorm_inf(), qr);
    }
  }
}

// ------------------------------------- pipe-PR-CG without recomputing w
// The ablation of Section 3.2 (Eq. 3.23, Fig. 2): w_k is never recomputed as
// A r~_k but carried as w'_k = w_{k-1} - alpha_{k-1} u_{k-1}, and under Jacobi
// w~_k as w~'_k = w~_{k-1} - alpha_{k-1} M^{-1} u_{k-1}, so each sweep forms
// the single product u_{k-1} = A s~_{k-1}.  The carried w and w~ live in
// V.w[0] and V.u[0] (each row reads and rewrites only its own entry); every
// other step is k_pipe's.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_pipe_nr(Op op, Pc pc, Vecs V, DevState* S,
                                                    double* partials, int qr, int qw) {
  if (__ldcg(&S->done)) return;
  const double alpha = __ldcg(&S->alpha);
  const double beta = __ldcg(&S->beta);
  const double* __restrict__ rt_o = Pc::on ? V.rt[qr] : V.r[qr];
  const double* __restrict__ st_o = Pc::on ? V.st[qr] : V.s[qr];
  const double* __restrict__ r_o = V.r[qr];
  const double* __restrict__ s_o = V.s[qr];
  double* __restrict__ x = V.x;
  double* __restrict__ p = V.p[0];
  double* __restrict__ w = V.w[0];
  double* __restrict__ wt = V.u[0];
  const double ad = std::is_same<Pc, PcScalar>::value ? alpha * pc(0) : 0.0;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  PRCG_ROWS(i, op.n) {
    const double u = op.row(i, [&](int j) { return __ldg(st_o + j); });
    const double si = __ldg(s_o + i);
    x[i] = fma(alpha, p[i], x[i]);
    const double rn = fma(-alpha, si, __ldg(r_o + i));
    const double wp = fma(-alpha, u, w[i]);
    w[i] = wp;
    double rtn = rn, sn, stn;
    if (Pc::on) {
      const double sti = __ldg(st_o + i);
      rtn = fma(-alpha, sti, __ldg(rt_o + i));
      const double wtp = sub_scaled(pc, i, alpha, ad, u, wt[i]);
      wt[i] = wtp;
      sn = fma(beta, si, wp);
      stn = fma(beta, sti, wtp);
      V.rt[qw][i] = rtn;
      V.st[qw][i] = stn;
    } else {
      sn = fma(beta, si, wp);
      stn = sn;
    }
    const double pn = fma(beta, p[i], rtn);
    p[i] = pn;
    V.r[qw][i] = rn;
    V.s[qw][i] = sn;
    acc[0] = fma(pn, sn, acc[0]);
    acc[1] = fma(rtn, sn, acc[1]);
    acc[2] = fma(stn, sn, acc[2]);
    if (Pc::on) acc[3] = fma(rtn, rn, acc[3]);
    acc[4] = fma(rn, rn, acc[4]);
  }
  double tot[5];
  if (grid_sum<5>(acc, partials, S, tot) && threadIdx.x == 0) {
    const int k = S->k + 1;
    S->mu = tot[0];
    S->sigma = tot[1];
    S->gamma = tot[2];
    S->nu = Pc::on ? tot[3] : tot[4];
    S->rho = tot[4];
    trace_pr_sums(S, k);
    if (!record_and_test(S, k, tot[4])) scalar_step_pr(S, false);
  }
}

// ------------------------------------------------------- CG-CG (Appendix E)
// Scalars of the Chronopoulos-Gear / Ghysels-Vanroose recurrences, formed by
// the last CTA after the reduction of nu_k, eta_k, <r_k, r_k> (the order of
// Appendix E: stopping test, beta_k, mu_k = eta_k - (beta_k / alpha_{k-1}) nu_k,
// alpha_k).
__device__ __forceinline__ void scalar_step_cg(DevState* S, int k, double nu, double eta,
                                               double rho) {
  S->rho = rho;
  S->eta = eta;
  trace(S, k, TR_NU, nu);
  trace(S, k, TR_ETA, eta);
  trace(S, k, TR_RHO, rho);
  if (record_and_test(S, k, rho)) return;
  if (!finite(nu) || !(nu > 0.0)) { breakdown(S); return; }
  const double beta = nu / S->nu;
  const double mu = eta - (beta / S->alpha) * nu;
  if (!finite(mu) || !(mu > 0.0)) { breakdown(S); return; }
  S->beta = beta;
  S->mu = mu;
  S->nu = nu;
  S->alpha = nu / mu;
  trace(S, k, TR_BETA, beta);
  trace(S, k, TR_MU, mu);
  trace(S, k + 1, TR_ALPHA, S->alpha);
}

// Sweep A of CG-CG iteration k: finish iteration k-1 (p_{k-1} = r~_{k-1} +
// beta p, s_{k-1} = w_{k-1} + beta s), then x_k, r_k and r~_k = M^{-1} r_k.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_cg_a(Op op, Pc pc, Vecs V, DevState* S) {
  if (__ldcg(&S->done)) return;
  const double alpha = __ldcg(&S->alpha);
  const double beta = __ldcg(&S->beta);
  double* __restrict__ x = V.x;
  double* __restrict__ r = V.r[0];
  double* __restrict__ rt = Pc::on ? V.rt[0] : V.r[0];
  double* __restrict__ p = V.p[0];
  double* __restrict__ s = V.s[0];
  const double* __restrict__ w = V.w[0];
  PRCG_ROWS(i, op.n) {
    const double pn = fma(beta, p[i], rt[i]);
    const double sn = fma(beta, s[i], __ldg(w + i));
    p[i] = pn;
    s[i] = sn;
    x[i] = fma(alpha, pn, x[i]);
    const double rn = fma(-alpha, sn, r[i]);
    r[i] = rn;
    if (Pc::on) V.rt[0][i] = pc(i) * rn;
  }
}

// Sweep B of CG-CG iteration k: w_k = A r~_k, nu_k, eta_k = <r~_k, w_k>, <r_k, r_k>.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_cg_b(Op op, Pc pc, Vecs V, DevState* S,
                                                 double* partials) {
  if (__ldcg(&S->done)) return;
  const double* __restrict__ rt = Pc::on ? V.rt[0] : V.r[0];
  const double* __restrict__ r = V.r[0];
  double acc[3] = {0.0, 0.0, 0.0};
  PRCG_ROWS(i, op.n) {
    const double wn = op.row(i, [&](int j) { return __ldg(rt + j); });
    V.w[0][i] = wn;
    const double rti = __ldg(rt + i), ri = __ldg(r + i);
    if (Pc::on) acc[0] = fma(rti, ri, acc[0]);   // unpreconditioned: nu_k = <r_k, r_k>
    acc[1] = fma(rti, wn, acc[1]);
    acc[2] = fma(ri, ri, acc[2]);
  }
  double tot[3];
  if (grid_sum<3>(acc, partials, S, tot) && threadIdx.x == 0)
    scalar_step_cg(S, S->k + 1, Pc::on ? tot[0] : tot[2], tot[1], tot[2]);
}

// --------------------------------------------------- GV-CG (Appendix E)
// One sweep per iteration k: t_{k-1} = A M^{-1} w_{k-1} from the stored
// w_{k-1} (buffer qr), the updates that finish iteration k-1 (p, s, s~,
// u with beta_{k-1}), the updates of iteration k (x_k, r_k, r~_k by
// recurrence, w_k = w_{k-1} - alpha u_{k-1}, to buffer qw) and nu_k, eta_k.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_gv(Op op, Pc pc, Vecs V, DevState* S,
                                               double* partials, int qr, int qw) {
  if (__ldcg(&S->done)) return;
  const double alpha = __ldcg(&S->alpha);
  const double beta = __ldcg(&S->beta);
  const double* __restrict__ w_o = V.w[qr];
  double* __restrict__ x = V.x;
  double* __restrict__ r = V.r[0];
  double* __restrict__ p = V.p[0];
  double* __restrict__ s = V.s[0];
  double* __restrict__ u = V.u[0];
  double acc[3] = {0.0, 0.0, 0.0};
  PRCG_ROWS(i, op.n) {
    const double t = op.row(i, [&](int j) {
      const double wj = __ldg(w_o + j);
      return Pc::on ? pc(j) * wj : wj;
    });
    const double wi = __ldg(w_o + i);
    const double rti = Pc::on ? V.rt[0][i] : r[i];
    const double pn = fma(beta, p[i], rti);
    const double sn = fma(beta, s[i], wi);
    const double un = fma(beta, u[i], t);
    double stn = sn;
    if (Pc::on) stn = fma(beta, V.st[0][i], pc(i) * wi);
    p[i] = pn;
    s[i] = sn;
    u[i] = un;
    x[i] = fma(alpha, pn, x[i]);
    const double rn = fma(-alpha, sn, r[i]);
    r[i] = rn;
    double rtn = rn;
    if (Pc::on) {
      V.st[0][i] = stn;
      rtn = fma(-alpha, stn, rti);
      V.rt[0][i] = rtn;
    }
    const double wn = fma(-alpha, un, wi);
    V.w[qw][i] = wn;
    if (Pc::on) acc[0] = fma(rtn, rn, acc[0]);   // unpreconditioned: nu_k = <r_k, r_k>
    acc[1] = fma(rtn, wn, acc[1]);
    acc[2] = fma(rn, rn, acc[2]);
  }
  double tot[3];
  if (grid_sum<3>(acc, partials, S, tot) && threadIdx.x == 0)
    scalar_step_cg(S, S->k + 1, Pc::on ? tot[0] : tot[2], tot[1], tot[2]);
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

// ||e||_A^2 = e^T A e with e = x* - x (x* in V.t, x in V.w[1]) into S->eta:
// the error measure of the paper's convergence study (Section 4).
template <class Op>
__global__ void __launch_bounds__(kBlock) k_anorm(Op op, Vecs V, DevState* S, double* partials) {
  double acc[1] = {0.0};
  const double* __restrict__ xs = V.t;
  const double* __restrict__ xx = V.w[1];
  PRCG_ROWS(i, op.n) {
    const double ae = op.row(i, [&](int j) { return __ldg(xs + j) - __ldg(xx + j); });
    acc[0] = fma(__ldg(xs + i) - __ldg(xx + i), ae, acc[0]);
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, S, tot) && threadIdx.x == 0) S->eta = tot[0];
}

}  // namespace prcg
