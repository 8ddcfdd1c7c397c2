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
