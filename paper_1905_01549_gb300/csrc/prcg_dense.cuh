// Products with a dense symmetric matrix (DenseOp, prcg_ops.cuh).
//
// A is stored column-major with a leading dimension that is a multiple of 32
// (for symmetric A this is also row-major).  The product y = A v is split
// into warp units: unit (g, c) is the 32 rows 32g .. 32g+31 against column
// block c.  Lane l owns row 32g + l, so each step of the unit's column loop
// is one coalesced 256-byte load of A; v_j is the same for every lane (a
// broadcast load).  Each lane adds its column block in column order and
// writes the partial part[c][i]; DenseOp::row() adds the ncb partials of a
// row in block order, so the product is fixed by (n, ncb) alone.
//
// On GB300 this product is bound by FP64 issue rather than HBM: one FMA per
// 8 bytes of A needs 0.85 T FMA/s at the measured 6.78 TB/s, and the FP64
// pipe delivers 2 FMA per SM per clock (0.63 T/s at 2.07 GHz).  The paired
// product [A s~, A r~] of pipe-PR-CG reads A once but doubles the FMAs, so
// it costs about twice the single product here.
#pragma once

#include "prcg_ops.cuh"

namespace prcg {

// The vector a product is formed with: v_j = a_j (DS_PLAIN), scale_j * a_j
// (DS_SCALE: Jacobi's M^{-1} w of GV-CG) or a_j - sub_j (DS_SUB: the error
// x* - x of prcg_error_anorm).  The form is a template argument: as a
// run-time choice the compiler if-converts it into FP64 instructions on
// every element, tripling the FP64 issue of the product.  Loads are coherent
// (L2): inside the persistent solve the vector was written by other CTAs in
// the same launch.
enum DenseSrcMode { DS_PLAIN = 0, DS_SCALE = 1, DS_SUB = 2 };

struct DenseSrc {
  const double* a = nullptr;
  const double* scale = nullptr;
  const double* sub = nullptr;
  template <int MODE>
  __device__ __forceinline__ double at(int j) const {
    double v = __ldcg(a + j);
    if constexpr (MODE == DS_SCALE) v = __ldcg(scale + j) * v;
    if constexpr (MODE == DS_SUB) v = v - __ldcg(sub + j);
    return v;
  }
};

// Units gw, gw + nw, ... of the product(s) with s0 (and s1 when NV == 2).
template <int NV, int MODE>
__device__ __forceinline__ void dense_units(const DenseOp& op, const DenseSrc& s0,
                                            const DenseSrc& s1, int gw, int nw) {
  const int lane = threadIdx.x & 31;
  const int ng = (op.n + 31) >> 5;
  const int units = ng * op.ncb;
  for (int u = gw; u < units; u += nw) {
    const int g = u % ng, c = u / ng;
    const int i = (g << 5) + lane;
    if (i >= op.n) continue;
    const int j0 = c * op.cbw;
    const int j1 = min(op.n, j0 + op.cbw);
    const double* col = op.A + (size_t)j0 * op.lda + i;
    double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
    for (int j = j0; j < j1; ++j) {
      const double aij = __ldcs(col);   // streamed: A is read once per product
      col += op.lda;
      a0 = fma(aij, s0.template at<MODE>(j), a0);
      if (NV == 2) a1 = fma(aij, s1.template at<MODE>(j), a1);
    }
    op.part0[(size_t)c * op.n + i] = a0;
    if (NV == 2) op.part1[(size_t)c * op.n + i] = a1;
  }
}

// Stand-alone product launched before a sweep of the graph / host loop
// paths.  With check_done the launch is a no-op once the run has finished
// (the sweeps after convergence inside the last loop body).
template <int NV, int MODE>
__global__ void __launch_bounds__(kBlock) k_dense_product(DenseOp op, DevState* S, DenseSrc s0,
                                                          DenseSrc s1, int check_done) {
  if (check_done && __ldcg(&S->done)) return;
  dense_units<NV, MODE>(op, s0, s1, (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5),
                  (int)((gridDim.x * blockDim.x) >> 5));
}

}  // namespace prcg
