// TMA staging of the SELL-32 entry stream for the matrix-product sweeps.
//
// A tile is 256 consecutive rows = 8 slices, whose column indices and values
// are contiguous in the SELL-32 arrays (slices are stored back to back and
// every slice start is a multiple of 32 entries, so both byte offsets are
// 128-byte aligned and every size is a multiple of 16 bytes).  One thread
// moves a whole tile's entries into shared memory with two cp.async.bulk
// copies completing on a "full" mbarrier; while the CTA computes tile m,
// tile m+1 is in flight (two stages; three in the pipelined sweep).  Warps
// release a stage on its "empty" mbarrier and the copying thread refills it
// once all have, so warps never meet at a CTA-wide barrier between tiles.
// The rows' own vector entries and the gathered columns still go through
// ordinary loads.  Every wait on an mbarrier is bounded: after kTmaSpinLimit
// polls the kernel records PRCG_ERR_TIMEOUT in the scalar block, waits
// (bounded) for its copies in flight and returns.
#pragma once

#include "prcg_kernels.cuh"

namespace prcg {

constexpr int kTmaRows = kBlock;            // rows per tile (one per thread)
constexpr int kTmaCap = kTmaRows * 7;       // entries per stage (tiles of <= 7 per row on average)
// Stages of the copy pipeline: two for the single-product sweeps; three for
// the pipelined sweep, whose longer per-tile arithmetic (two products and
// the updates of Algorithm 3) leaves more time to hide -- measured at 256^3:
// k_pipe_tma 886 -> 850 us with three, while k_pr_b_tma slowed 354 -> 449 us
// (fewer resident CTAs for the same shared memory).
constexpr int kTmaStages = 2;
constexpr int kTmaStagesPipe = 3;
constexpr long kTmaSpinLimit = 1L << 24;

template <int ST>
struct __align__(128) TmaSmemT {
  int col[ST][kTmaCap];
  double val[ST][kTmaCap];
  unsigned long long bar[ST];     // "full": the stage's copies have landed
  unsigned long long empty[ST];   // every warp is done with the stage
  int failed;
};
using TmaSmem = TmaSmemT<kTmaStages>;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count = 1) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// true once the barrier's phase with the given parity has completed
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (long it = 0; it < kTmaSpinLimit; ++it)
    if (mbar_test(bar, parity)) return true;
  return false;
}

// Issue the entry copy of `tile` into `stage` (one thread).
template <int ST>
__device__ __forceinline__ void tma_issue(TmaSmemT<ST>& sm, const SellOp& op, int tile, int stage) {
  const int s0 = tile * (kTmaRows / 32);
  const int nsl = (op.n + 31) / 32;
  const int s1 = min(s0 + kTmaRows / 32, nsl);
  const int e0 = __ldg(op.sptr + s0), e1 = __ldg(op.sptr + s1);
  const unsigned cnt = (unsigned)(e1 - e0);
  mbar_expect_tx(&sm.bar[stage], cnt * 12u);   // a tile of empty rows completes at once
  if (cnt > 0) {
    bulk_g2s(sm.col[stage], op.scol + e0, cnt * 4u, &sm.bar[stage]);
    bulk_g2s(sm.val[stage], op.sval + e0, cnt * 8u, &sm.bar[stage]);
  }
}

// Run `row(i, visit)` for every row of this CTA's tiles with the tile's
// entries staged in shared memory; visit(f) calls f(j, a_ij) for the row's
// entries in stored order (padding entries included, as the SELL sweep does).
// Each warp waits for its tile's "full" barrier itself and, when done,
// arrives on the stage's "empty" barrier; thread 0 refills a stage once
// every warp has released it, so no warp waits for the slowest one between
// tiles.  Returns false if a wait timed out (the caller reports the error).
template <int ST, class RowFn>
__device__ __forceinline__ bool sell_tma_sweep(TmaSmemT<ST>& sm, const SellOp& op, RowFn&& row) {
  const int ntiles = (op.n + kTmaRows - 1) / kTmaRows;
  const int tid = threadIdx.x, lane = tid & 31;
  volatile int* failed = &sm.failed;
  int issued[ST] = {};         // thread 0's bookkeeping of copies per stage
  if (tid == 0) {
    for (int q = 0; q < ST; ++q) {
      mbar_init(&sm.bar[q]);
      mbar_init(&sm.empty[q], blockDim.x >> 5);
    }
    sm.failed = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < ST; ++q) {
      const int t = blockIdx.x + q * gridDim.x;
      if (t < ntiles) {
        tma_issue(sm, op, t, q);
        ++issued[q];
      }
    }
  }
  int consumed = 0;   // tiles whose "full" phase thread 0 has observed
  int m = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++m) {
    const int stage = m % ST;
    const unsigned parity = (unsigned)((m / ST) & 1);
    const bool landed = mbar_wait_bounded(&sm.bar[stage], parity);
    const int stop = __shfl_sync(0xffffffffu, lane == 0 ? *failed : 0, 0);
    if (!__all_sync(0xffffffffu, landed) || stop) {   // warp-uniform decision
      if (lane == 0) *failed = 1;
      break;
    }
    if (tid == 0) ++consumed;
    const int i = t * kTmaRows + tid;
    if (i < op.n) {
      const int sl = i >> 5;
      const int tile_e0 = __ldg(op.sptr + t * (kTmaRows / 32));
      const int off = __ldg(op.sptr + sl) - tile_e0 + (i & 31);
      const int L = __ldg(op.slen + sl);
      const int* __restrict__ cs = sm.col[stage];
      const double* __restrict__ vs = sm.val[stage];
      row(i, [&](auto&& f) {
        for (int e = 0; e < L; ++e) f(cs[off + 32 * e], vs[off + 32 * e]);
      });
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[stage]);   // this warp is done with the stage
    if (tid == 0) {
      const int tn = t + ST * gridDim.x;
      if (tn < ntiles) {
        if (mbar_wait_bounded(&sm.empty[stage], parity)) {
          fence_proxy_async();
          tma_issue(sm, op, tn, stage);
          ++issued[stage];
        } else {
          *failed = 1;
        }
      }
    }
  }
  __syncthreads();
  const bool ok = sm.failed == 0;
  if (!ok && tid == 0) {
    // drain (bounded) every copy issued but not yet observed, before exit
    int total = 0;
    for (int q = 0; q < ST; ++q) total += issued[q];
    for (int mm = consumed; mm < total; ++mm)
      mbar_wait_bounded(&sm.bar[mm % ST], (unsigned)((mm / ST) & 1));
  }
  __syncthreads();
  return ok;
}

// ------------------------------------------------- sweeps with staged entries
// Same arithmetic and order as k_hs_c / k_pr_b / k_pipe (prcg_kernels.cuh).

__device__ __forceinline__ void tma_fail(DevState* S) {
  S->status = -4;   // PRCG_ERR_TIMEOUT
  S->done = 1;
}

template <class Pc>
__global__ void __launch_bounds__(kBlock) k_hs_c_tma(SellOp op, Pc pc, Vecs V, DevState* S,
                                                     double* partials) {
  if (__ldcg(&S->done)) return;
  __shared__ TmaSmem sm;
  double acc[1] = {0.0};
  const double* __restrict__ p = V.p[0];
  const bool ok = sell_tma_sweep(sm, op, [&](int i, auto&& visit) {
    double sn = 0.0;
    visit([&](int j, double a) { sn = fma(a, __ldg(p + j), sn); });
    V.s[0][i] = sn;
    acc[0] = fma(__ldg(p + i), sn, acc[0]);
  });
  if (!ok) {
    if (threadIdx.x == 0) tma_fail(S);
    return;
  }
  double tot[1];
  if (grid_sum<1>(acc, partials, S, tot) && threadIdx.x == 0) {
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

template <class Pc>
__global__ void __launch_bounds__(kBlock) k_pr_b_tma(SellOp op, Pc pc, Vecs V, DevState* S,
                                                     double* partials, const double* partials_a,
                                                     int grid_a, int meurant) {
  if (__ldcg(&S->done)) return;
  __shared__ TmaSmem sm;
  const double* __restrict__ p = V.p[0];
  const double* __restrict__ rt = Pc::on ? V.rt[0] : V.r[0];
  double acc[3] = {0.0, 0.0, 0.0};
  const bool ok = sell_tma_sweep(sm, op, [&](int i, auto&& visit) {
    double sn = 0.0;
    visit([&](int j, double a) { sn = fma(a, __ldg(p + j), sn); });
    V.s[0][i] = sn;
    acc[0] = fma(__ldg(p + i), sn, acc[0]);
    acc[1] = fma(__ldg(rt + i), sn, acc[1]);
    // gamma_k = <d s_k, s_k>; a constant d is factored out of the sum
    if (std::is_same<Pc, PcVec>::value)
      acc[2] = fma(pc(i) * sn, sn, acc[2]);
    else
      acc[2] = fma(sn, sn, acc[2]);
  });
  if (!ok) {
    if (threadIdx.x == 0) tma_fail(S);
    return;
  }
  double tot[3];
  if (!grid_sum<3>(acc, partials, S, tot)) return;
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
    if (!record_and_test(S, k, rho)) scalar_step_pr(S, meurant != 0);
  }
}

template <class Pc>
__global__ void __launch_bounds__(kBlock) k_pipe_tma(SellOp op, Pc pc, Vecs V, DevState* S,
                                                     double* partials, int qr, int qw, int meurant) {
  if (__ldcg(&S->done)) return;
  __shared__ TmaSmemT<kTmaStagesPipe> sm;
  const double alpha = __ldcg(&S->alpha);
  const double beta = __ldcg(&S->beta);
  const double* __restrict__ rt_o = Pc::on ? V.rt[qr] : V.r[qr];
  const double* __restrict__ st_o = Pc::on ? V.st[qr] : V.s[qr];
  const double* __restrict__ r_o = V.r[qr];
  const double* __restrict__ s_o = V.s[qr];
  double* __restrict__ x = V.x;
  double* __restrict__ p = V.p[0];
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const bool ok = sell_tma_sweep(sm, op, [&](int i, auto&& visit) {
    double u = 0.0, w = 0.0;
    visit([&](int j, double a) {
      u = fma(a, __ldg(st_o + j), u);
      w = fma(a, __ldg(rt_o + j), w);
    });
    const double si = __ldg(s_o + i);
    x[i] = fma(alpha, p[i], x[i]);
    const double rn = fma(-alpha, si, __ldg(r_o + i));
    const double wp = fma(-alpha, u, w);
    double rtn = rn, sn, stn;
    if (Pc::on) {
      const double sti = __ldg(st_o + i);
      rtn = fma(-alpha, sti, __ldg(rt_o + i));
      const double wtp = wt_pred(pc, i, wp);
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
    if (Pc::on) acc[3] = fma(rtn, rn, acc[3]);   // unpreconditioned: nu_k = rho_k
    acc[4] = fma(rn, rn, acc[4]);
  });
  if (!ok) {
    if (threadIdx.x == 0) tma_fail(S);
    return;
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
    if (!record_and_test(S, k, tot[4])) scalar_step_pr(S, meurant != 0);
  }
}

// Largest number of entries of any 256-row tile (host check at set-up).
inline bool sell_fits_tma(const int* h_sptr, int nslices) {
  for (int s0 = 0; s0 < nslices; s0 += kTmaRows / 32) {
    const int s1 = s0 + kTmaRows / 32 < nslices ? s0 + kTmaRows / 32 : nslices;
    if (h_sptr[s1] - h_sptr[s0] > kTmaCap) return false;
  }
  return true;
}

}  // namespace prcg
