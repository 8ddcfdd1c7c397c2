// Host-side launch of the fused sweeps for one (operator, preconditioner)
// pair.  Each prcg_inst_*.cu file instantiates this for its operator so the
// library compiles in parallel translation units.
#pragma once

#include "prcg_persistent.cuh"
#include "prcg_tma.cuh"
#include "prcg_mixed.cuh"

namespace prcg {

enum Phase {
  PH_INIT_A = 0,
  PH_INIT_B = 1,
  PH_HS_A = 2,
  PH_HS_B = 3,
  PH_HS_C = 4,
  PH_PR_A = 5,
  PH_PR_B = 6,
  PH_PIPE = 7,
  PH_TRUE_RES = 8,
  PH_MX_RESID = 9,
  PH_MX_INIT_A = 10,
  PH_MX_INIT_B = 11,
  PH_MX_PR_A = 12,
  PH_MX_PR_B = 13,
  PH_MX_UPDATE = 14,
  PH_CG_A = 15,
  PH_CG_B = 16,
  PH_GV = 17,
  PH_PERSIST = 18,  // the whole solve as one cooperative launch (all but the ablations)
  PH_ANORM = 19,    // ||x* - x||_A^2 (x* in V.t, x in V.w[1]) into S->eta
  PH_PIPE_NR = 20   // pipe-PR-CG with w carried instead of recomputed (ablation)
};

struct Plan {
  OpDesc op;
  PcDesc pc;
  Vecs v;
  DevState* S;
  double* partials;
  double* partials_a;    // PR sweep A's per-CTA sums
  int sms;
  // mixed precision: FP32 vectors, the inner solve's scalar block and the
  // scalar argument of the phase being launched (1 / ||t|| or ||t||)
  Vecs32 w;
  DevState* S2;
  double arg;
  GridBar* gb;   // grid barrier of the persistent solve
};

// Cooperative launch of the persistent solve: one CTA per SM.
template <class Op, class Pc, int VARIANT>
cudaError_t launch_persist(const Plan& P, int meurant, cudaStream_t st) {
  auto k = k_persist<Op, Pc, VARIANT>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kPersistThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1 || P.sms > kMaxPersistCtas) return cudaErrorCooperativeLaunchTooLarge;
  Op op(P.op);
  Pc pc(P.pc);
  Vecs v = P.v;
  DevState* S = P.S;
  double* partials = P.partials;
  GridBar* gb = P.gb;
  void* args[] = {(void*)&op, (void*)&pc, (void*)&v, (void*)&S, (void*)&partials, (void*)&gb,
                  (void*)&meurant};
  return cudaLaunchCooperativeKernel((const void*)k, dim3(P.sms), dim3(kPersistThreads), args, 0, st);
}

using LaunchFn = cudaError_t (*)(const Plan&, int phase, int variant, int qr, int qw,
                                 cudaStream_t);

// CTAs for a sweep: enough to fill every SM at the kernel's occupancy, but
// never more tiles than rows.
template <class K>
inline int grid_for(K kernel, int n, int sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  long tiles = ((long)n + kBlock - 1) / kBlock;
  long g = (long)per_sm * sms;
  if (g > tiles) g = tiles;
  if (g > kMaxGrid) g = kMaxGrid;
  if (g < 1) g = 1;
  return (int)g;
}

// FP32 inner-solve phases; operators without an FP32 row are not supported.
template <class Op, class = void>
struct HasRow32 : std::false_type {};
template <class Op>
struct HasRow32<Op, decltype((void)&Op::template row32<float (*)(int)>)> : std::true_type {};

template <class Op, class Pc>
cudaError_t launch_mixed(const Plan& P, int phase, cudaStream_t st) {
  if constexpr (!HasRow32<Op>::value) {
    return cudaErrorNotSupported;
  } else {
    Op op(P.op);
    Pc pc(P.pc);
    const int n = P.op.n;
    double* pa = P.partials_a;
    switch (phase) {
      case PH_MX_INIT_A: {
        auto k = k_mx_init_a<Op, Pc>;
        k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.w, P.S2, P.partials);
        break;
      }
      case PH_MX_INIT_B: {
        auto k = k_mx_init_b<Op, Pc>;
        k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.w, P.S2, P.partials);
        break;
      }
      case PH_MX_PR_A: {
        auto k = k_mx_pr_a<Op, Pc>;
        k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.w, P.S2, pa);
        break;
      }
      case PH_MX_PR_B: {
        auto k = k_mx_pr_b<Op, Pc>;
        const int grid_a = grid_for(k_mx_pr_a<Op, Pc>, n, P.sms);
        k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.w, P.S2, P.partials, pa, grid_a);
        break;
      }
      case PH_MX_UPDATE: {
        auto k = k_mx_update<Op, Pc>;
        k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, P.v, P.w, P.arg);
        break;
      }
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
}

// Dense operators: form the product a sweep needs before launching it (the
// sweep's row() then reads the partial products).  No-op for other operators.
template <class Op, class Pc>
cudaError_t dense_prepass(const Plan& P, const Op& op, int phase, int qr, cudaStream_t st) {
  if constexpr (!IsDense<Op>::value) {
    return cudaSuccess;
  } else {
    const Vecs& V = P.v;
    DenseSrc s0, s1;
    int nv = 1, check = 1;
    switch (phase) {
      case PH_INIT_A: s0.a = V.x; break;
      case PH_INIT_B:
      case PH_HS_C:
      case PH_PR_B: s0.a = V.p[0]; break;
      case PH_PIPE:
        s0.a = Pc::on ? V.st[qr] : V.s[qr];
        s1.a = Pc::on ? V.rt[qr] : V.r[qr];
        nv = 2;
        break;
      case PH_CG_B: s0.a = Pc::on ? V.rt[0] : V.r[0]; break;
      case PH_PIPE_NR: s0.a = Pc::on ? V.st[qr] : V.s[qr]; break;
      case PH_GV:
        s0.a = V.w[qr];
        if (Pc::on) s0.scale = P.pc.d;
        break;
      case PH_TRUE_RES: s0.a = V.x; check = 0; break;
      case PH_ANORM:
        s0.a = V.t;
        s0.sub = V.w[1];
        check = 0;
        break;
      default: return cudaSuccess;
    }
    const long units = (long)((op.n + 31) / 32) * op.ncb;
    long g = (units + kBlock / 32 - 1) / (kBlock / 32);
    if (g > (long)P.sms * 8) g = (long)P.sms * 8;
    if (nv == 2)
      k_dense_product<2, DS_PLAIN><<<(int)g, kBlock, 0, st>>>(op, P.S, s0, s1, check);
    else if (s0.scale)
      k_dense_product<1, DS_SCALE><<<(int)g, kBlock, 0, st>>>(op, P.S, s0, s1, check);
    else if (s0.sub)
      k_dense_product<1, DS_SUB><<<(int)g, kBlock, 0, st>>>(op, P.S, s0, s1, check);
    else
      k_dense_product<1, DS_PLAIN><<<(int)g, kBlock, 0, st>>>(op, P.S, s0, s1, check);
    return cudaGetLastError();
  }
}

template <class Op, class Pc>
cudaError_t launch_phase(const Plan& P, int phase, int variant, int qr, int qw, cudaStream_t st) {
  Op op(P.op);
  Pc pc(P.pc);
  const int n = P.op.n;
  if (phase != PH_PERSIST) {
    const cudaError_t e = dense_prepass<Op, Pc>(P, op, phase, qr, st);
    if (e != cudaSuccess) return e;
  }
  const int meurant = (variant == V_M || variant == V_PIPE_M) ? 1 : 0;
  switch (phase) {
    case PH_INIT_A: {
      auto k = k_init_a<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials);
      break;
    }
    case PH_INIT_B: {
      auto k = k_init_b<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials, variant);
      break;
    }
    case PH_HS_A: {
      auto k = k_hs_a<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials);
      break;
    }
    case PH_HS_B: {
      auto k = k_hs_b<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S);
      break;
    }
    case PH_HS_C: {
      if constexpr (std::is_same<Op, SellOp>::value) {
        if (P.op.tma) {
          auto kt = k_hs_c_tma<Pc>;
          kt<<<grid_for(kt, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials);
          break;
        }
      }
      auto k = k_hs_c<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials);
      break;
    }
    case PH_PR_A: {
      auto k = k_pr_a<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials_a);
      break;
    }
    case PH_PR_B: {
      const int grid_a = grid_for(k_pr_a<Op, Pc>, n, P.sms);
      if constexpr (std::is_same<Op, SellOp>::value) {
        if (P.op.tma) {
          auto kt = k_pr_b_tma<Pc>;
          kt<<<grid_for(kt, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials, P.partials_a,
                                                         grid_a, meurant);
          break;
        }
      }
      auto k = k_pr_b<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials, P.partials_a,
                                                   grid_a, meurant);
      break;
    }
    case PH_PIPE: {
      if constexpr (std::is_same<Op, SellOp>::value) {
        if (P.op.tma) {
          auto kt = k_pipe_tma<Pc>;
          kt<<<grid_for(kt, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials, qr, qw,
                                                         meurant);
          break;
        }
      }
      auto k = k_pipe<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials, qr, qw, meurant);
      break;
    }
    case PH_PIPE_NR: {
      auto k = k_pipe_nr<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials, qr, qw);
      break;
    }
    case PH_CG_A: {
      auto k = k_cg_a<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S);
      break;
    }
    case PH_CG_B: {
      auto k = k_cg_b<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials);
      break;
    }
    case PH_GV: {
      auto k = k_gv<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials, qr, qw);
      break;
    }
    case PH_PERSIST:
      if (variant == V_HS) return launch_persist<Op, Pc, V_HS>(P, 0, st);
      if (variant == V_PR || variant == V_M) return launch_persist<Op, Pc, V_PR>(P, meurant, st);
      if (variant == V_PIPE || variant == V_PIPE_M) return launch_persist<Op, Pc, V_PIPE>(P, meurant, st);
      if (variant == V_CGCG) return launch_persist<Op, Pc, V_CGCG>(P, 0, st);
      if (variant == V_GV) return launch_persist<Op, Pc, V_GV>(P, 0, st);
      return cudaErrorInvalidValue;
    case PH_TRUE_RES: {
      auto k = k_true_res<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials);
      break;
    }
    case PH_ANORM: {
      auto k = k_anorm<Op>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, P.v, P.S, P.partials);
      break;
    }
    case PH_MX_RESID: {
      auto k = k_mx_resid<Op, Pc>;
      k<<<grid_for(k, n, P.sms), kBlock, 0, st>>>(op, pc, P.v, P.S, P.partials);
      break;
    }
    case PH_MX_INIT_A:
    case PH_MX_INIT_B:
    case PH_MX_PR_A:
    case PH_MX_PR_B:
    case PH_MX_UPDATE:
      return launch_mixed<Op, Pc>(P, phase, st);
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Launchers exported by the instantiation units.
cudaError_t launch_csr(const Plan&, int, int, int, int, cudaStream_t);
LaunchFn launcher_for(int op_kind, int pc_kind);

}  // namespace prcg
