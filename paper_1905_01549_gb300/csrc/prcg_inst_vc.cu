// Instantiation of the fused sweeps for variable-coefficient 5/7-point stencils.
#include "prcg_launch.cuh"

namespace prcg {

LaunchFn launcher_vc(int op_kind, int pc_kind) {
  if (op_kind == OP_VC2 && pc_kind == PC_NONE) return &launch_phase<VarStencilOp<2>, PcNone>;
  if (op_kind == OP_VC2 && pc_kind == PC_VEC) return &launch_phase<VarStencilOp<2>, PcVec>;
  if (op_kind == OP_VC3 && pc_kind == PC_NONE) return &launch_phase<VarStencilOp<3>, PcNone>;
  if (op_kind == OP_VC3 && pc_kind == PC_VEC) return &launch_phase<VarStencilOp<3>, PcVec>;
  return nullptr;
}

}  // namespace prcg
