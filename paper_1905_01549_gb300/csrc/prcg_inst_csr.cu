// Instantiation of the fused sweeps for sparse matrices (CSR and SELL-32).
#include "prcg_launch.cuh"

namespace prcg {

LaunchFn launcher_csr(int op_kind, int pc_kind) {
  if (op_kind == OP_CSR && pc_kind == PC_NONE) return &launch_phase<CsrOp, PcNone>;
  if (op_kind == OP_CSR && pc_kind == PC_VEC) return &launch_phase<CsrOp, PcVec>;
  if (op_kind == OP_SELL && pc_kind == PC_NONE) return &launch_phase<SellOp, PcNone>;
  if (op_kind == OP_SELL && pc_kind == PC_VEC) return &launch_phase<SellOp, PcVec>;
  return nullptr;
}

}  // namespace prcg

static_assert(prcg::HasRow32<prcg::SellOp>::value, "SELL-32 has an FP32 row");
static_assert(!prcg::HasRow32<prcg::CsrOp>::value, "CSR has no FP32 row");
