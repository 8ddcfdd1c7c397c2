// Instantiation of the fused sweeps for constant-coefficient 5/7-point stencils.
#include "prcg_launch.cuh"

namespace prcg {

LaunchFn launcher_st(int op_kind, int pc_kind) {
  if (op_kind == OP_ST2 && pc_kind == PC_NONE) return &launch_phase<StencilOp<2>, PcNone>;
  if (op_kind == OP_ST2 && pc_kind == PC_SCALAR) return &launch_phase<StencilOp<2>, PcScalar>;
  if (op_kind == OP_ST3 && pc_kind == PC_NONE) return &launch_phase<StencilOp<3>, PcNone>;
  if (op_kind == OP_ST3 && pc_kind == PC_SCALAR) return &launch_phase<StencilOp<3>, PcScalar>;
  return nullptr;
}

}  // namespace prcg

static_assert(prcg::HasRow32<prcg::StencilOp<3>>::value, "stencil has an FP32 row");
