// Instantiation of the fused sweeps for sparse matrices whose Jacobi
// diagonal is one constant (d_i = d for every row, e.g. constant-coefficient
// Poisson stored as CSR): d is then a scalar, as for the constant stencils.
#include "prcg_launch.cuh"

namespace prcg {

LaunchFn launcher_csr_scalar(int op_kind, int pc_kind) {
  if (op_kind == OP_CSR && pc_kind == PC_SCALAR) return &launch_phase<CsrOp, PcScalar>;
  if (op_kind == OP_SELL && pc_kind == PC_SCALAR) return &launch_phase<SellOp, PcScalar>;
  return nullptr;
}

}  // namespace prcg
