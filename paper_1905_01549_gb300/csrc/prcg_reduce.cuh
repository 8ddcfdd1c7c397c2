// Deterministic CTA-level sums of a few doubles, shared by every kernel of
// the library (the on-chip half of the paper's global reduction, Table 1
// C_gr).  The order of additions depends only on the launch shape, so
// reruns are bitwise identical.
#pragma once

#include <cuda_runtime.h>

namespace prcg {

// Warp reduce-scatter of v[0..C) (C slots per lane, the same in every lane).
// While C > 1, a halving step keeps half of the slots in each lane -- the low
// half where lane bit O is clear, the high half where it is set -- and adds
// the partner lane's copy of that half; once one slot is left the remaining
// steps are a plain butterfly.  A lane so spends about NV + 4 FP64 adds
// instead of 5 NV.  That matters here: the FP64 pipe issues two lanes per
// clock per SM, so every warp-wide FP64 add costs 16 issue cycles.  On
// return v[0] of a lane holds the warp total of value `base` if real > 0;
// lanes that differ only in the butterfly bits hold equal values.
template <int C, int O, int NV>
__device__ __forceinline__ void warp_rs(double (&v)[NV], int lane, int& base, int& real) {
  if constexpr (O > 0) {
    if constexpr (C > 1) {
      constexpr int H = (C + 1) / 2;
      const bool up = (lane & O) != 0;
#pragma unroll
      for (int j = 0; j < H; ++j) {
        const double hi = (H + j < C) ? v[H + j] : 0.0;
        const double keep = up ? hi : v[j];
        const double send = up ? v[j] : hi;
        v[j] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      if (up) {
        base += H;
        real = real > H ? real - H : 0;
      } else {
        real = real < H ? real : H;
      }
      warp_rs<H, O / 2>(v, lane, base, real);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
      warp_rs<1, O / 2>(v, lane, base, real);
    }
  }
}

// Lanes that write the totals after warp_rs: one per group of equal lanes.
template <int NV>
__host__ __device__ constexpr int rs_writer_mask() {
  return NV <= 1 ? 31 : NV <= 2 ? 15 : NV <= 4 ? 7 : 3;
}

// Reduce v over the warp; lane `writer` lanes store total m to out[m * stride].
template <int NV>
__device__ __forceinline__ void warp_sum_store(double (&v)[NV], double* out, int stride) {
  const int lane = threadIdx.x & 31;
  int base = 0, real = NV;
  warp_rs<NV, 16>(v, lane, base, real);
  if (real > 0 && (lane & rs_writer_mask<NV>()) == 0) out[base * stride] = v[0];
}

// Sum v[0..NV) over the CTA in a fixed order; the result is valid in thread 0.
// `warp_active` (uniform within each warp) marks warps that may hold nonzero
// values; the others skip the shuffles and contribute exact zeros.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm, bool warp_active = true) {
  static_assert(NV >= 1 && NV <= 8, "1..8 sums");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  __syncthreads();  // sm may still be read by a previous call
  if (warp_active)
    warp_sum_store<NV>(v, sm + wid, 32);
  else if (lane < NV)
    sm[lane * 32 + wid] = 0.0;
  __syncthreads();
  if (wid == 0) {
    double t[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) t[m] = lane < nwarps ? sm[m * 32 + lane] : 0.0;
    __syncwarp();
    warp_sum_store<NV>(t, sm, 32);
    __syncwarp();
    if (lane == 0) {
#pragma unroll
      for (int m = 0; m < NV; ++m) v[m] = sm[m * 32];
    }
  }
}

}  // namespace prcg
