// Persistent whole-solve kernels for small and medium systems.
//
// Below a few million rows a sweep moves so little data that a CG iteration
// is dominated by the cost of its synchronisations -- kernel boundaries and
// last-CTA reductions -- which is the paper's C_gr argument on one GPU.  The
// persistent form runs initialize() and the whole iteration loop as one
// cooperative launch of one CTA per SM; every CTA owns a fixed block of rows,
// and the iteration's data dependencies are grid barriers:
//   HS-CG    3 barriers per iteration (reduction, p complete, reduction)
//   PR-CG    2 barriers per iteration (p complete, reduction); M-CG alike
//   CG-CG    2 barriers per iteration (r~ complete, reduction)
//   pipe-PR  1 barrier per iteration  (the reduction); pipe-M-CG alike
//   GV-CG    1 barrier per iteration  (the reduction)
// -- the synchronisation counts of the paper's Table 1 (dense operators add
// one barrier per product, after the in-kernel product).
// At a reducing barrier every CTA adds all CTAs' partial sums itself, in CTA
// order, so every CTA forms the same scalars from bitwise-identical totals,
// takes identical control decisions and meets the same barriers.  Waiting
// CTAs poll the arrival counter a bounded number of times; on expiry the CTA
// records PRCG_ERR_TIMEOUT and every CTA leaves the loop at its next
// barrier.  The cooperative launch guarantees that all CTAs are resident.
#pragma once

#include "prcg_dense.cuh"
#include "prcg_kernels.cuh"

namespace prcg {

constexpr int kPersistThreads = 1024;
constexpr long kBarrierSpinLimit = 1L << 22;

// Barrier state, written by the host before each launch.  The arrival
// counter only grows (barrier e completes when it reaches (e + 1) *
// gridDim.x), so no CTA ever resets it; the error flag sits on its own
// 128-byte line.  spin_limit bounds every wait (polls); skip_cta / skip_epoch
// are a failure-injection hook for tests: that CTA does not arrive at that
// barrier, so every CTA's wait there runs out (-1: off).
struct GridBar {
  alignas(128) unsigned count;
  alignas(128) int err;
  long long spin_limit;
  int skip_cta;
  int skip_epoch;
};

constexpr int kMaxPersistCtas = 256;   // >= the SM count (one CTA per SM)

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Arrive at barrier `epoch` and wait, bounded, for every CTA (thread 0 only,
// after a __syncthreads).  The arrival is a release and the poll an acquire
// at GPU scope, so the CTA's writes before the barrier are visible to every
// CTA after it.  Returns false once the wait has expired or another CTA has
// given up.
__device__ __forceinline__ bool barrier_arrive_wait(GridBar* gb, unsigned epoch) {
  if (!(gb->skip_cta == (int)blockIdx.x && gb->skip_epoch == (int)epoch)) {
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&gb->count) : "memory");
  }
  const unsigned target = (epoch + 1u) * gridDim.x;
  const long limit = gb->spin_limit;
  long it = 0;
  while (ld_acquire_u32(&gb->count) < target) {
    if ((++it & 1023) == 0 && (it > limit || *(volatile int*)&gb->err)) {
      gb->err = 1;
      return false;
    }
  }
  return true;
}

// What warp 0 decides after a reducing barrier and every thread then reads.
struct Bcast {
  double d[3];
  int status;   // kRunning or a final status
};

// Grid barrier with grid totals of v.  Each CTA writes its partial sums
// (buffer epoch & 1, so a CTA that races ahead to the next barrier never
// overwrites sums still being read), arrives and waits; then warp m of every
// CTA adds value m of all CTAs in one round of independent loads and a fixed
// tree, so every CTA forms bitwise-identical totals.  Warp 0 alone then runs
// `step(tot, out)` -- the scalar step: an FP64 division costs hundreds of
// cycles and the FP64 pipe issues two lanes per clock per SM, so forming the
// scalars redundantly in all 32 warps would cost several microseconds --
// and every thread receives `out`.  `epoch` counts the barriers passed
// (identical in all CTAs); `warp_active` is block_sum's.  Returns false once
// a wait has expired.
template <int NV, class Step>
__device__ __forceinline__ bool grid_sync_sum(double (&v)[NV], double* partials, GridBar* gb,
                                              unsigned& epoch, bool warp_active, Bcast& out,
                                              Step&& step) {
  static_assert(NV >= 1 && NV <= 8, "1..8 sums");
  static_assert(kMaxPersistCtas == 256, "partials are gathered in 8 loads per lane");
  __shared__ double sm[NV * 32];
  __shared__ double s_tot[NV];
  __shared__ Bcast s_out;
  __shared__ int s_ok;
  const int G = gridDim.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* buf = partials + (size_t)(epoch & 1) * kMaxPersistCtas * 8;
  block_sum<NV>(v, sm, warp_active);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int m = 0; m < NV; ++m) buf[blockIdx.x * 8 + m] = v[m];
    s_ok = barrier_arrive_wait(gb, epoch) ? 1 : 0;
  }
  __syncthreads();
  if (wid < NV) {
    double t[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int b = lane + 32 * j;
      t[j] = b < G ? __ldcg(&buf[b * 8 + wid]) : 0.0;
    }
    double a = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if (lane == 0) s_tot[wid] = a;
    if (NV > 1) asm volatile("bar.sync 1, %0;" ::"r"(NV * 32) : "memory");
    if (wid == 0) {
      double tot[NV];
#pragma unroll
      for (int m = 0; m < NV; ++m) tot[m] = s_tot[m];
      Bcast o{{0.0, 0.0, 0.0}, kRunning};
      step(tot, o);
      if (lane == 0) s_out = o;
    }
  }
  __syncthreads();
  out = s_out;
  ++epoch;
  return s_ok != 0;
}

// Plain grid barrier (no sums).
__device__ __forceinline__ bool grid_sync(GridBar* gb, unsigned& epoch) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) s_ok = barrier_arrive_wait(gb, epoch) ? 1 : 0;
  __syncthreads();
  ++epoch;
  return s_ok != 0;
}

// Rows of this CTA: a contiguous block, its start a multiple of 32 (so a
// warp's 32 consecutive rows form one SELL-32 slice).
struct RowBlock {
  int begin, end;
  __device__ RowBlock(int n) {
    const int per = ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
    begin = min(n, (int)blockIdx.x * per);
    end = min(n, begin + per);
  }
};

#define PRCG_OWN_ROWS(i, rb) for (int i = (rb).begin + threadIdx.x; i < (rb).end; i += blockDim.x)

// Scalar step of the predict-and-recompute variants (run by warp 0):
// alpha_k = nu_k / mu_k, nu'_{k+1} by Eq. 2.3 (or Meurant's form), beta.
__device__ __forceinline__ void pr_scalars(double nu, double mu, double sigma, double gamma,
                                           bool meurant, Bcast& o) {
  if (!finite(nu) || !finite(mu) || !(mu > 0.0) || nu < 0.0) {
    o.status = 2;
    return;
  }
  const double alpha = nu / mu;
  const double np = meurant ? -nu + alpha * alpha * gamma
                            : nu - 2.0 * alpha * sigma + alpha * alpha * gamma;
  if (!finite(np) || np < 0.0 || nu == 0.0) {
    o.status = 2;
    return;
  }
  o.d[0] = alpha;
  o.d[1] = np / nu;
  o.d[2] = np;
}

// Scalar step of CG-CG / GV-CG (Appendix E) after the reduction of
// nu_k, eta_k, rho_k (run by warp 0): the stopping test, beta_k =
// nu_k / nu_{k-1}, mu_k = eta_k - (beta_k / alpha_{k-1}) nu_k, alpha_k.
// o.d = {alpha_k, beta_k, nu_k}.
__device__ __forceinline__ void cg_scalars(DevState* S, int k, double nu, double eta, double rho,
                                           double nu_prev, double alpha_prev, double stop2,
                                           int maxit, Bcast& q);

// Trace writes of the persistent solve: the first thread of CTA 0 only.
__device__ __forceinline__ void ptrace(const DevState* S, int k, int f, double v) {
  if (blockIdx.x == 0 && threadIdx.x == 0) trace(S, k, f, v);
}

__device__ __forceinline__ void ptrace_pr_step(const DevState* S, int k, const Bcast& q) {
  if (q.status != kRunning) return;
  ptrace(S, k + 1, TR_ALPHA, q.d[0]);
  ptrace(S, k + 1, TR_BETA, q.d[1]);
  ptrace(S, k + 1, TR_NU_PRED, q.d[2]);
}

// Stopping test of iteration k, ||r_k||^2 <= tol^2 ||b||^2 (no square root or
// division on the critical path); the first thread records rho_k, which the
// host turns into ||r_k|| / ||b||.  Returns the final status or kRunning.
__device__ __forceinline__ int stop_test(DevState* S, int k, double rho, double stop2, int maxit) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && S->hist) S->hist[k] = rho;
  if (rho <= stop2) return 0;
  if (k >= maxit) return 1;
  return kRunning;
}

__device__ __forceinline__ void cg_scalars(DevState* S, int k, double nu, double eta, double rho,
                                           double nu_prev, double alpha_prev, double stop2,
                                           int maxit, Bcast& q) {
  ptrace(S, k, TR_NU, nu);
  ptrace(S, k, TR_ETA, eta);
  ptrace(S, k, TR_RHO, rho);
  q.status = stop_test(S, k, rho, stop2, maxit);
  if (q.status != kRunning) return;
  if (!finite(nu) || !(nu > 0.0)) {
    q.status = 2;
    return;
  }
  const double beta = nu / nu_prev;
  const double mu = eta - (beta / alpha_prev) * nu;
  if (!finite(mu) || !(mu > 0.0)) {
    q.status = 2;
    return;
  }
  q.d[0] = nu / mu;
  q.d[1] = beta;
  q.d[2] = nu;
  ptrace(S, k, TR_BETA, beta);
  ptrace(S, k, TR_MU, mu);
  ptrace(S, k + 1, TR_ALPHA, q.d[0]);
}

__device__ __forceinline__ void finish(DevState* S, int k, int status) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S->k = k;
    S->status = status;
    S->done = 1;
  }
}

constexpr int kZeroRhs = -101;   // internal: b == 0

// The Jacobi vector of a preconditioner, or NULL (GV-CG's dense product of
// M^{-1} w).
template <class Pc>
__device__ __forceinline__ const double* pc_vector(const Pc&) {
  return nullptr;
}
__device__ __forceinline__ const double* pc_vector(const PcVec& p) { return p.d; }

// Dense operators: every warp of the grid forms its units of the product
// with v0 (and v1), then a barrier makes the partials visible to the row
// loop that follows.  Other operators gather inside the row loop: no-op.
template <class Op>
__device__ __forceinline__ bool persist_product(const Op& op, const double* v0, const double* v1,
                                                GridBar* gb, unsigned& epoch,
                                                const double* scale = nullptr) {
  if constexpr (IsDense<Op>::value) {
    DenseSrc s0, s1;
    s0.a = v0;
    s0.scale = scale;
    s1.a = v1;
    const int gw = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    const int nw = (int)(gridDim.x * (blockDim.x >> 5));
    if (v1)
      dense_units<2, DS_PLAIN>(op, s0, s1, gw, nw);
    else if (scale)
      dense_units<1, DS_SCALE>(op, s0, s1, gw, nw);
    else
      dense_units<1, DS_PLAIN>(op, s0, s1, gw, nw);
    return grid_sync(gb, epoch);
  } else {
    return true;
  }
}

// One persistent solve.  VARIANT: V_HS, V_PR (meurant -> M-CG), V_PIPE
// (meurant -> pipe-PR-M-CG), V_CGCG, V_GV.
template <class Op, class Pc, int VARIANT>
__global__ void __launch_bounds__(kPersistThreads, 1)
    k_persist(Op op, Pc pc, Vecs V, DevState* S, double* partials, GridBar* gb, int meurant) {
  // Jacobi with a constant d (a scalar) or a vector d
  constexpr bool kScalarD = std::is_same<Pc, PcScalar>::value;
  constexpr bool kVecD = Pc::on && !kScalarD;
  constexpr bool kNuDot = kVecD;   // HS: nu_k = <d r_k, r_k> needs its own sum
  const RowBlock rb(op.n);
  // warps that own rows; the others add nothing to the reductions
  const bool wact = rb.begin + (int)(threadIdx.x & ~31u) < rb.end;
  unsigned epoch = 0;
  const double tol2 = S->tol2;
  const int maxit = S->maxit;
  double* __restrict__ x = V.x;
  Bcast o;
  // ---- initialize(): r_0, r~_0, p_0; nu_0, rho_0, <b, b>
  if (!persist_product(op, x, nullptr, gb, epoch)) {
    finish(S, 0, -4);
    return;
  }
  double a3[3] = {0.0, 0.0, 0.0};
  PRCG_OWN_ROWS(i, rb) {
    const double ax = op.row(i, [&](int j) { return __ldcg(x + j); });
    const double bi = __ldg(V.b + i);
    const double r = bi - ax;
    const double rt = Pc::on ? pc(i) * r : r;
    V.r[0][i] = r;
    if (Pc::on) V.rt[0][i] = rt;
    V.p[0][i] = rt;
    a3[0] = fma(rt, r, a3[0]);
    a3[1] = fma(r, r, a3[1]);
    a3[2] = fma(bi, bi, a3[2]);
  }
  // o.d = {nu_0, tol^2 ||b||^2}
  if (!grid_sync_sum<3>(a3, partials, gb, epoch, wact, o, [&](const double* t, Bcast& q) {
        const double bn2 = t[2];
        q.d[0] = t[0];
        q.d[1] = tol2 * bn2;
        ptrace(S, 0, TR_NU, t[0]);
        ptrace(S, 0, TR_RHO, t[1]);
        if (blockIdx.x == 0 && threadIdx.x == 0) S->bnorm2 = bn2;
        if (bn2 == 0.0) {
          if (blockIdx.x == 0 && threadIdx.x == 0) {
            S->zero_rhs = 1;
            if (S->hist) S->hist[0] = 0.0;
          }
          q.status = kZeroRhs;
        } else {
          q.status = stop_test(S, 0, t[1], q.d[1], maxit);
        }
      })) {
    finish(S, 0, -4);
    return;
  }
  if (o.status != kRunning) {
    finish(S, 0, o.status == kZeroRhs ? 0 : o.status);
    return;
  }
  double nu = o.d[0];
  const double stop2 = o.d[1];
  // s_0 = A p_0 (s~_0 stored for pipe), mu_0, sigma_0, gamma_0
  {
    const double* p0 = V.p[0];
    if (!persist_product(op, p0, nullptr, gb, epoch)) {
      finish(S, 0, -4);
      return;
    }
    double b3[3] = {0.0, 0.0, 0.0};
    PRCG_OWN_ROWS(i, rb) {
      const double s = op.row(i, [&](int j) { return __ldcg(p0 + j); });
      const double st = Pc::on ? pc(i) * s : s;
      V.s[0][i] = s;
      if ((VARIANT == V_PIPE || VARIANT == V_GV) && Pc::on) V.st[0][i] = st;
      if (VARIANT == V_CGCG || VARIANT == V_GV) V.w[0][i] = s;   // w_0 = A r~_0 = s_0 (p_0 = r~_0)
      if (VARIANT == V_GV) V.u[0][i] = 0.0;   // multiplied by beta_0 = 0 in the first sweep
      const double rt = Pc::on ? V.rt[0][i] : V.r[0][i];
      b3[0] = fma(p0[i], s, b3[0]);
      b3[1] = fma(rt, s, b3[1]);
      b3[2] = fma(st, s, b3[2]);
    }
    if (!grid_sync_sum<3>(b3, partials, gb, epoch, wact, o, [&](const double* t, Bcast& q) {
          ptrace(S, 0, TR_MU, t[0]);
          ptrace(S, 0, TR_SIGMA, t[1]);
          ptrace(S, 0, TR_GAMMA, t[2]);
          if (VARIANT == V_HS || VARIANT == V_CGCG || VARIANT == V_GV) {
            // alpha_0; CG-CG / GV-CG start with beta_0 = 0 (o.d[1] stays 0)
            if (!finite(nu) || !finite(t[0]) || !(t[0] > 0.0) || nu < 0.0) {
              q.status = 2;
            } else {
              q.d[0] = nu / t[0];
              ptrace(S, 1, TR_ALPHA, q.d[0]);
            }
          } else {
            pr_scalars(nu, t[0], t[1], t[2], meurant != 0, q);
            ptrace_pr_step(S, 0, q);
          }
        })) {
      finish(S, 0, -4);
      return;
    }
    if (o.status != kRunning) {
      finish(S, 0, o.status);
      return;
    }
  }
  double alpha = o.d[0], beta = o.d[1];
  // ---- the iteration loop
  for (int k = 1; k <= maxit; ++k) {
    if (VARIANT == V_HS) {
      // A: x_k, r_k; nu_k, rho_k -> beta_k
      double a2[2] = {0.0, 0.0};
      PRCG_OWN_ROWS(i, rb) {
        x[i] = fma(alpha, V.p[0][i], x[i]);
        const double rn = fma(-alpha, V.s[0][i], V.r[0][i]);
        V.r[0][i] = rn;
        // nu_k = <d r_k, r_k>: with a constant d, d <r_k, r_k> (no
        // preconditioner: nu_k = rho_k)
        if (kNuDot) a2[0] = fma(pc(i) * rn, rn, a2[0]);
        a2[1] = fma(rn, rn, a2[1]);
      }
      if (!grid_sync_sum<2>(a2, partials, gb, epoch, wact, o, [&](const double* t, Bcast& q) {
            const double nun = kNuDot ? t[0] : (kScalarD ? pc(0) * t[1] : t[1]);
            ptrace(S, k, TR_NU, nun);
            ptrace(S, k, TR_RHO, t[1]);
            q.status = stop_test(S, k, t[1], stop2, maxit);
            if (q.status != kRunning) return;
            if (!finite(nun) || !(nun > 0.0)) {
              q.status = 2;
              return;
            }
            q.d[0] = nun / nu;   // beta_k
            q.d[1] = nun;        // nu_k
            ptrace(S, k, TR_BETA, q.d[0]);
          })) {
        finish(S, k, -4);
        return;
      }
      if (o.status != kRunning) {
        finish(S, k, o.status);
        return;
      }
      beta = o.d[0];
      nu = o.d[1];
      // B: p_k
      PRCG_OWN_ROWS(i, rb) {
        const double ri = V.r[0][i];
        V.p[0][i] = fma(beta, V.p[0][i], Pc::on ? pc(i) * ri : ri);
      }
      if (!grid_sync(gb, epoch)) {
        finish(S, k, -4);
        return;
      }
      // C: s_k = A p_k, mu_k -> alpha_k
      const double* pp = V.p[0];
      if (!persist_product(op, pp, nullptr, gb, epoch)) {
        finish(S, k, -4);
        return;
      }
      double c1[1] = {0.0};
      bool paired = false;
      if constexpr (HasRows2<Op>::value) {
        if (op.pairs_ok()) {
          auto g = [&](int j) { return __ldcg(pp + j); };
          auto g2 = [&](int j) { return __ldcg(reinterpret_cast<const double2*>(pp + j)); };
          for (int i = rb.begin + 2 * (int)threadIdx.x; i < rb.end; i += 2 * (int)blockDim.x) {
            const double2 s2 = op.rows2(i, g, g2);
            *reinterpret_cast<double2*>(V.s[0] + i) = s2;
            const double2 p2 = *reinterpret_cast<const double2*>(pp + i);
            c1[0] = fma(p2.x, s2.x, c1[0]);
            c1[0] = fma(p2.y, s2.y, c1[0]);
          }
          paired = true;
        }
      }
      if (!paired) {
        PRCG_OWN_ROWS(i, rb) {
          const double sn = op.row(i, [&](int j) { return __ldcg(pp + j); });
          V.s[0][i] = sn;
          c1[0] = fma(pp[i], sn, c1[0]);
        }
      }
      if (!grid_sync_sum<1>(c1, partials, gb, epoch, wact, o, [&](const double* t, Bcast& q) {
            ptrace(S, k, TR_MU, t[0]);
            if (!finite(t[0]) || !(t[0] > 0.0)) {
              q.status = 2;
            } else {
              q.d[0] = nu / t[0];
              ptrace(S, k + 1, TR_ALPHA, q.d[0]);
            }
          })) {
        finish(S, k, -4);
        return;
      }
      if (o.status != kRunning) {
        finish(S, k, o.status);
        return;
      }
      alpha = o.d[0];
    } else if (VARIANT == V_PR) {
      // A: x_k, r_k, r~_k, p_k; partial nu_k, rho_k
      double a5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      const double ad = std::is_same<Pc, PcScalar>::value ? alpha * pc(0) : 0.0;
      PRCG_OWN_ROWS(i, rb) {
        const double si = V.s[0][i], pi = V.p[0][i];
        x[i] = fma(alpha, pi, x[i]);
        const double rn = fma(-alpha, si, V.r[0][i]);
        V.r[0][i] = rn;
        double rtn = rn;
        if (Pc::on) {
          rtn = sub_scaled(pc, i, alpha, ad, si, V.rt[0][i]);
          V.rt[0][i] = rtn;
        }
        V.p[0][i] = fma(beta, pi, rtn);
        if (Pc::on) a5[0] = fma(rtn, rn, a5[0]);   // unpreconditioned: nu_k = rho_k
        a5[1] = fma(rn, rn, a5[1]);
      }
      if (!grid_sync(gb, epoch)) {
        finish(S, k, -4);
        return;
      }
      // B: s_k = A p_k; mu_k, sigma_k, gamma_k
      const double* pp = V.p[0];
      const double* rtv = Pc::on ? V.rt[0] : V.r[0];
      if (!persist_product(op, pp, nullptr, gb, epoch)) {
        finish(S, k, -4);
        return;
      }
      bool paired = false;
      if constexpr (HasRows2<Op>::value) {
        if (op.pairs_ok()) {
          // two rows of one grid line per thread (the block starts on a
          // multiple of 32 rows and n is even)
          auto g = [&](int j) { return __ldcg(pp + j); };
          auto g2 = [&](int j) { return __ldcg(reinterpret_cast<const double2*>(pp + j)); };
          for (int i = rb.begin + 2 * (int)threadIdx.x; i < rb.end; i += 2 * (int)blockDim.x) {
            const double2 s2 = op.rows2(i, g, g2);
            *reinterpret_cast<double2*>(V.s[0] + i) = s2;
            const double2 p2 = *reinterpret_cast<const double2*>(pp + i);
            const double2 r2 = *reinterpret_cast<const double2*>(rtv + i);
            a5[2] = fma(p2.x, s2.x, a5[2]);
            a5[3] = fma(r2.x, s2.x, a5[3]);
            a5[4] = fma(kVecD ? pc(i) * s2.x : s2.x, s2.x, a5[4]);
            a5[2] = fma(p2.y, s2.y, a5[2]);
            a5[3] = fma(r2.y, s2.y, a5[3]);
            a5[4] = fma(kVecD ? pc(i + 1) * s2.y : s2.y, s2.y, a5[4]);
          }
          paired = true;
        }
      }
      if (!paired) {
        PRCG_OWN_ROWS(i, rb) {
          const double sn = op.row(i, [&](int j) { return __ldcg(pp + j); });
          V.s[0][i] = sn;
          a5[2] = fma(pp[i], sn, a5[2]);
          a5[3] = fma(rtv[i], sn, a5[3]);
          a5[4] = fma(kVecD ? pc(i) * sn : sn, sn, a5[4]);
        }
      }
      if (!grid_sync_sum<5>(a5, partials, gb, epoch, wact, o, [&](const double* t, Bcast& q) {
            ptrace(S, k, TR_NU, Pc::on ? t[0] : t[1]);
            ptrace(S, k, TR_RHO, t[1]);
            ptrace(S, k, TR_MU, t[2]);
            ptrace(S, k, TR_SIGMA, t[3]);
            // gamma_k = <d s_k, s_k>: a constant d is factored out of the sum
            const double gam = kScalarD ? pc(0) * t[4] : t[4];
            ptrace(S, k, TR_GAMMA, gam);
            q.status = stop_test(S, k, t[1], stop2, maxit);
            if (q.status != kRunning) return;
            pr_scalars(Pc::on ? t[0] : t[1], t[2], t[3], gam, meurant != 0, q);
            ptrace_pr_step(S, k, q);
          })) {
        finish(S, k, -4);
        return;
      }
      if (o.status != kRunning) {
        finish(S, k, o.status);
        return;
      }
      alpha = o.d[0];
      beta = o.d[1];
    } else if (VARIANT == V_PIPE) {
      // pipe: u_{k-1}, w_{k-1} from buffer qr, updates of iteration k to qw
      const int qr = (k - 1) & 1, qw = k & 1;
      const double* rt_o = Pc::on ? V.rt[qr] : V.r[qr];
      const double* st_o = Pc::on ? V.st[qr] : V.s[qr];
      const double* r_o = V.r[qr];
      const double* s_o = V.s[qr];
      if (!persist_product(op, st_o, rt_o, gb, epoch)) {
        finish(S, k, -4);
        return;
      }
      double a5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      PRCG_OWN_ROWS(i, rb) {
        double u, w;
        op.row2(i, [&](int j) { return __ldcg(st_o + j); }, [&](int j) { return __ldcg(rt_o + j); },
                u, w);
        const double si = s_o[i];
        const double pi = V.p[0][i];
        x[i] = fma(alpha, pi, x[i]);
        const double rn = fma(-alpha, si, r_o[i]);
        const double wp = fma(-alpha, u, w);
        double rtn = rn, sn, stn;
        if (Pc::on) {
          const double sti = st_o[i];
          rtn = fma(-alpha, sti, rt_o[i]);
          const double wtp = wt_pred(pc, i, wp);
          sn = fma(beta, si, wp);
          stn = fma(beta, sti, wtp);
          V.rt[qw][i] = rtn;
          V.st[qw][i] = stn;
        } else {
          sn = fma(beta, si, wp);
          stn = sn;
        }
        const double pn = fma(beta, pi, rtn);
        V.p[0][i] = pn;
        V.r[qw][i] = rn;
        V.s[qw][i] = sn;
        a5[0] = fma(pn, sn, a5[0]);
        a5[1] = fma(rtn, sn, a5[1]);
        a5[2] = fma(stn, sn, a5[2]);
        if (Pc::on) a5[3] = fma(rtn, rn, a5[3]);   // unpreconditioned: nu_k = rho_k
        a5[4] = fma(rn, rn, a5[4]);
      }
      if (!grid_sync_sum<5>(a5, partials, gb, epoch, wact, o, [&](const double* t, Bcast& q) {
            ptrace(S, k, TR_MU, t[0]);
            ptrace(S, k, TR_SIGMA, t[1]);
            ptrace(S, k, TR_GAMMA, t[2]);
            const double nuk = Pc::on ? t[3] : t[4];
            ptrace(S, k, TR_NU, nuk);
            ptrace(S, k, TR_RHO, t[4]);
            q.status = stop_test(S, k, t[4], stop2, maxit);
            if (q.status != kRunning) return;
            pr_scalars(nuk, t[0], t[1], t[2], meurant != 0, q);
            ptrace_pr_step(S, k, q);
          })) {
        finish(S, k, -4);
        return;
      }
      if (o.status != kRunning) {
        finish(S, k, o.status);
        return;
      }
      alpha = o.d[0];
      beta = o.d[1];
    } else if (VARIANT == V_CGCG) {
      // A: finish iteration k-1 (p, s with beta_{k-1}), then x_k, r_k and
      // r~_k = M^{-1} r_k (row-local)
      PRCG_OWN_ROWS(i, rb) {
        const double rti = Pc::on ? V.rt[0][i] : V.r[0][i];
        const double pn = fma(beta, V.p[0][i], rti);
        const double sn = fma(beta, V.s[0][i], V.w[0][i]);
        V.p[0][i] = pn;
        V.s[0][i] = sn;
        x[i] = fma(alpha, pn, x[i]);
        const double rn = fma(-alpha, sn, V.r[0][i]);
        V.r[0][i] = rn;
        if (Pc::on) V.rt[0][i] = pc(i) * rn;
      }
      if (!grid_sync(gb, epoch)) {
        finish(S, k, -4);
        return;
      }
      // B: w_k = A r~_k; nu_k, eta_k = <r~_k, w_k>, rho_k
      const double* rtv = Pc::on ? V.rt[0] : V.r[0];
      if (!persist_product(op, rtv, nullptr, gb, epoch)) {
        finish(S, k, -4);
        return;
      }
      double a3[3] = {0.0, 0.0, 0.0};
      PRCG_OWN_ROWS(i, rb) {
        const double wn = op.row(i, [&](int j) { return __ldcg(rtv + j); });
        V.w[0][i] = wn;
        const double rti = rtv[i], ri = V.r[0][i];
        if (Pc::on) a3[0] = fma(rti, ri, a3[0]);   // unpreconditioned: nu_k = rho_k
        a3[1] = fma(rti, wn, a3[1]);
        a3[2] = fma(ri, ri, a3[2]);
      }
      if (!grid_sync_sum<3>(a3, partials, gb, epoch, wact, o, [&](const double* t, Bcast& q) {
            cg_scalars(S, k, Pc::on ? t[0] : t[2], t[1], t[2], nu, alpha, stop2, maxit, q);
          })) {
        finish(S, k, -4);
        return;
      }
      if (o.status != kRunning) {
        finish(S, k, o.status);
        return;
      }
      alpha = o.d[0];
      beta = o.d[1];
      nu = o.d[2];
    } else {
      // GV-CG: t_{k-1} = A M^{-1} w_{k-1} from buffer qr, the updates that
      // finish iteration k-1 (p, s, s~, u with beta_{k-1}), those of iteration
      // k (x_k, r_k, r~_k, w_k to buffer qw) and nu_k, eta_k, rho_k
      const int qr = (k - 1) & 1, qw = k & 1;
      const double* w_o = V.w[qr];
      if (!persist_product(op, w_o, nullptr, gb, epoch, pc_vector(pc))) {
        finish(S, k, -4);
        return;
      }
      double a3[3] = {0.0, 0.0, 0.0};
      PRCG_OWN_ROWS(i, rb) {
        const double t = op.row(i, [&](int j) {
          const double wj = __ldcg(w_o + j);
          return Pc::on ? pc(j) * wj : wj;
        });
        const double wi = w_o[i];
        const double rti = Pc::on ? V.rt[0][i] : V.r[0][i];
        const double pn = fma(beta, V.p[0][i], rti);
        const double sn = fma(beta, V.s[0][i], wi);
        const double un = fma(beta, V.u[0][i], t);
        double stn = sn;
        if (Pc::on) stn = fma(beta, V.st[0][i], pc(i) * wi);
        V.p[0][i] = pn;
        V.s[0][i] = sn;
        V.u[0][i] = un;
        x[i] = fma(alpha, pn, x[i]);
        const double rn = fma(-alpha, sn, V.r[0][i]);
        V.r[0][i] = rn;
        double rtn = rn;
        if (Pc::on) {
          V.st[0][i] = stn;
          rtn = fma(-alpha, stn, rti);
          V.rt[0][i] = rtn;
        }
        const double wn = fma(-alpha, un, wi);
        V.w[qw][i] = wn;
        if (Pc::on) a3[0] = fma(rtn, rn, a3[0]);   // unpreconditioned: nu_k = rho_k
        a3[1] = fma(rtn, wn, a3[1]);
        a3[2] = fma(rn, rn, a3[2]);
      }
      if (!grid_sync_sum<3>(a3, partials, gb, epoch, wact, o, [&](const double* t, Bcast& q) {
            cg_scalars(S, k, Pc::on ? t[0] : t[2], t[1], t[2], nu, alpha, stop2, maxit, q);
          })) {
        finish(S, k, -4);
        return;
      }
      if (o.status != kRunning) {
        finish(S, k, o.status);
        return;
      }
      alpha = o.d[0];
      beta = o.d[1];
      nu = o.d[2];
    }
  }
  finish(S, maxit, 1);
}

}  // namespace prcg
