// Instantiation of the sweeps for dense symmetric matrices (products formed
// by the column-block pre-pass of prcg_dense.cuh).
#include "prcg_launch.cuh"

namespace prcg {

LaunchFn launcher_dense(int op_kind, int pc_kind) {
  if (op_kind != OP_DENSE) return nullptr;
  if (pc_kind == PC_NONE) return &launch_phase<DenseOp, PcNone>;
  if (pc_kind == PC_VEC) return &launch_phase<DenseOp, PcVec>;
  return nullptr;
}

}  // namespace prcg

static_assert(!prcg::HasRow32<prcg::DenseOp>::value, "the dense operator has no FP32 row");
