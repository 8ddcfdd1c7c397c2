// The FP32 inner solve of the mixed-precision form (prcg_solve_f32_refined):
// FP32 vectors, compensated FP32 sums per thread, FP64 scalars, inside FP64
// iterative refinement.  Kept apart from the FP64 sweeps.
#pragma once

#include "prcg_kernels.cuh"

namespace prcg {

// The same for four rows (i a multiple of 4), rounded to FP32 for the
// mixed-precision inner solve.
template <class Pc>
__device__ __forceinline__ float4 pc_quad32(const Pc& pc, int i) {
  return make_float4((float)pc(i), (float)pc(i + 1), (float)pc(i + 2), (float)pc(i + 3));
}

// FP32 products of four consecutive rows i .. i+3 (i a multiple of 4) with
// the FP32 vector p, in the order row32() adds them.  Generic form: four
// gathered rows; the constant stencil overrides it (below).
template <class Op>
__device__ __forceinline__ float4 rows32x4(const Op& op, int i, const float* __restrict__ p) {
  auto g = [&](int j) { return __ldg(p + j); };
  return make_float4(op.row32(i, g), op.row32(i + 1, g), op.row32(i + 2, g), op.row32(i + 3, g));
}

__device__ __forceinline__ float4 pc_quad32(const PcVec& pc, int i) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(pc.d + i));
  const double2 b = __ldg(reinterpret_cast<const double2*>(pc.d + i + 2));
  return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

// Constant stencil, nx a multiple of 4: the four rows share y and z, so
// their neighbours are four aligned 16-byte loads (y and z neighbours, the
// rows themselves) and two scalars (the x neighbours outside the group).  A
// missing neighbour gets coefficient 0 as in row32(), which then adds
// 0 * p_i: the same FMA sequence, hence the same result.
template <int DIM>
__device__ __forceinline__ float4 rows32x4(const StencilOp<DIM>& op, int i,
                                           const float* __restrict__ p) {
  if (op.nx & 3) {
    auto g = [&](int j) { return __ldg(p + j); };
    return make_float4(op.row32(i, g), op.row32(i + 1, g), op.row32(i + 2, g), op.row32(i + 3, g));
  }
  const int nx = op.nx, ny = op.ny, nz = op.nz, pl = nx * ny;
  int x, y, z;
  op.coords(i, x, y, z);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto ld4 = [&](int j) { return __ldg(reinterpret_cast<const float4*>(p + j)); };
  const float4 c = ld4(i);
  const float lm = x > 0 ? __ldg(p + i - 1) : 0.f;
  const float rp = x + 4 < nx ? __ldg(p + i + 4) : 0.f;
  const float4 ym = y > 0 ? ld4(i - nx) : zero, yp = y < ny - 1 ? ld4(i + nx) : zero;
  const float4 zm = DIM == 3 && z > 0 ? ld4(i - pl) : zero;
  const float4 zp = DIM == 3 && z < nz - 1 ? ld4(i + pl) : zero;
  const float cym = y > 0 ? -1.f : 0.f, cyp = y < ny - 1 ? -1.f : 0.f;
  const float czm = z > 0 ? -1.f : 0.f, czp = z < nz - 1 ? -1.f : 0.f;
  const float cd = (float)op.cdiag;
  const float cv[4] = {c.x, c.y, c.z, c.w};
  const float ymv[4] = {ym.x, ym.y, ym.z, ym.w}, ypv[4] = {yp.x, yp.y, yp.z, yp.w};
  const float zmv[4] = {zm.x, zm.y, zm.z, zm.w}, zpv[4] = {zp.x, zp.y, zp.z, zp.w};
  float out[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int xq = x + q;
    float acc = 0.f;
    if (DIM == 3) acc = fmaf(czm, zmv[q], acc);
    acc = fmaf(cym, ymv[q], acc);
    acc = fmaf(xq > 0 ? -1.f : 0.f, q == 0 ? lm : cv[q - 1 < 0 ? 0 : q - 1], acc);
    acc = fmaf(cd, cv[q], acc);
    acc = fmaf(xq < nx - 1 ? -1.f : 0.f, q == 3 ? rp : cv[q + 1 > 3 ? 3 : q + 1], acc);
    acc = fmaf(cyp, ypv[q], acc);
    if (DIM == 3) acc = fmaf(czp, zpv[q], acc);
    out[q] = acc;
  }
  return make_float4(out[0], out[1], out[2], out[3]);
}

// ------------------------------------------------ mixed precision (FP32 inner)
// Iterative refinement: the outer loop forms t = b - A x in FP64, scales it
// to rhs = t / ||t|| in FP32, runs PR-CG on A d = rhs with FP32 vectors and
// FP32 matrix values (inner products: FP32 products, compensated FP32
// accumulation per thread, FP64 across threads; scalars alpha, beta, nu' in
// FP64, rounded to FP32 only where a vector update applies them), and adds
// x += ||t|| d in FP64.  S is the inner solve's own scalar block.

// FP64 outer residual t = b - A x with ||t||^2, ||b||^2 into S->eta, S->nu_pred.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_mx_resid(Op op, Pc pc, Vecs V, DevState* S,
                                                     double* partials) {
  double acc[2] = {0.0, 0.0};
  const double* __restrict__ x = V.x;
  PRCG_ROWS(i, op.n) {
    const double bi = __ldg(V.b + i);
    const double t = bi - op.row(i, [&](int j) { return __ldg(x + j); });
    V.t[i] = t;
    acc[0] = fma(t, t, acc[0]);
    acc[1] = fma(bi, bi, acc[1]);
  }
  double tot[2];
  if (grid_sum<2>(acc, partials, S, tot) && threadIdx.x == 0) {
    S->eta = tot[0];
    S->nu_pred = tot[1];
  }
}

// rhs = t * inv_norm in FP32, and the inner solve's initialize() for d_0 = 0:
// r_0 = rhs, r~_0 = M^{-1} r_0, p_0 = r~_0; nu_0, <r_0, r_0>, <rhs, rhs>.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_mx_init_a(Op op, Pc pc, Vecs V, Vecs32 W, DevState* S,
                                                      double* partials) {
  const double inv_norm = __ldcg(&S->arg);
  KahanF nu, rr;
  PRCG_ROWS(i, op.n) {
    const float ri = (float)(__ldg(V.t + i) * inv_norm);
    const float rti = Pc::on ? (float)pc(i) * ri : ri;
    W.rhs[i] = ri;
    W.r[i] = ri;
    W.rt[i] = rti;
    W.p[i] = rti;
    W.d[i] = 0.f;
    nu.add(rti * ri);
    rr.add(ri * ri);
  }
  double acc[2] = {nu.value(), rr.value()};
  double tot[2];
  if (grid_sum<2>(acc, partials, S, tot) && threadIdx.x == 0) {
    S->nu = tot[0];
    S->rho = tot[1];
    S->bnorm2 = tot[1];
    S->k = 0;
    record_and_test(S, 0, tot[1]);
  }
}

// s_0 = A p_0; mu_0, sigma_0, gamma_0; alpha_0, nu'_1, beta_1.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_mx_init_b(Op op, Pc pc, Vecs32 W, DevState* S,
                                                      double* partials) {
  if (__ldcg(&S->done)) return;
  KahanF mu, sg, ga;
  const float* __restrict__ p = W.p;
  PRCG_ROWS(i, op.n) {
    const float sn = op.row32(i, [&](int j) { return __ldg(p + j); });
    W.s[i] = sn;
    mu.add(__ldg(p + i) * sn);
    sg.add(__ldg(W.rt + i) * sn);
    ga.add((Pc::on ? (float)pc(i) * sn : sn) * sn);
  }
  double acc[3] = {mu.value(), sg.value(), ga.value()};
  double tot[3];
  if (grid_sum<3>(acc, partials, S, tot) && threadIdx.x == 0) {
    S->mu = tot[0];
    S->sigma = tot[1];
    S->gamma = tot[2];
    scalar_step_pr(S, false);
  }
}

// Sweep A of inner iteration k (FP32 vectors).
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_mx_pr_a(Op op, Pc pc, Vecs32 W, DevState* S,
                                                    double* partials_a) {
  if (__ldcg(&S->done)) return;
  const float af = (float)__ldcg(&S->alpha);
  const float bf = (float)__ldcg(&S->beta);
  KahanF nu, rr;
  // the update of one row; returns p_k and writes d, r, r~
  auto update = [&](float si, float pi, float& di, float& ri, float& rti, float dd) {
    di = fmaf(af, pi, di);
    const float rn = fmaf(-af, si, ri);
    ri = rn;
    float rtn = rn;
    if (Pc::on) {
      rtn = fmaf(-af, dd * si, rti);
      rti = rtn;
    }
    nu.add(rtn * rn);
    rr.add(rn * rn);
    return fmaf(bf, pi, rtn);
  };
  // four rows per thread with 16-byte accesses (FP32 vectors start on
  // 256-byte boundaries); the last CTA takes the n mod 4 remaining rows
  const int n = op.n, nq = n >> 2;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nq; j += gridDim.x * blockDim.x) {
    const int i = 4 * j;
    const float4 s4 = *reinterpret_cast<const float4*>(W.s + i);
    const float4 p4 = *reinterpret_cast<const float4*>(W.p + i);
    float4 d4 = *reinterpret_cast<const float4*>(W.d + i);
    float4 r4 = *reinterpret_cast<const float4*>(W.r + i);
    float4 rt4 = Pc::on ? *reinterpret_cast<const float4*>(W.rt + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 c4 = pc_quad32(pc, i);
    float4 pn;
    pn.x = update(s4.x, p4.x, d4.x, r4.x, rt4.x, c4.x);
    pn.y = update(s4.y, p4.y, d4.y, r4.y, rt4.y, c4.y);
    pn.z = update(s4.z, p4.z, d4.z, r4.z, rt4.z, c4.z);
    pn.w = update(s4.w, p4.w, d4.w, r4.w, rt4.w, c4.w);
    *reinterpret_cast<float4*>(W.d + i) = d4;
    *reinterpret_cast<float4*>(W.r + i) = r4;
    if (Pc::on) *reinterpret_cast<float4*>(W.rt + i) = rt4;
    *reinterpret_cast<float4*>(W.p + i) = pn;
  }
  if (blockIdx.x == gridDim.x - 1 && (int)threadIdx.x < n - 4 * nq) {
    const int i = 4 * nq + threadIdx.x;
    float di = W.d[i], ri = W.r[i], rti = Pc::on ? W.rt[i] : 0.f;
    W.p[i] = update(W.s[i], W.p[i], di, ri, rti, Pc::on ? (float)pc(i) : 1.f);
    W.d[i] = di;
    W.r[i] = ri;
    if (Pc::on) W.rt[i] = rti;
  }
  double acc[2] = {Pc::on ? nu.value() : rr.value(), rr.value()};
  __shared__ double sm[2 * 32];
  block_sum<2>(acc, sm);
  if (threadIdx.x == 0) {
    partials_a[blockIdx.x * 2 + 0] = acc[0];
    partials_a[blockIdx.x * 2 + 1] = acc[1];
  }
}

// Sweep B of inner iteration k: s_k = A p_k (FP32), mu, sigma, gamma; the
// reduction adds sweep A's sums and forms the next FP64 scalars.
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_mx_pr_b(Op op, Pc pc, Vecs32 W, DevState* S,
                                                    double* partials, const double* partials_a,
                                                    int grid_a) {
  if (__ldcg(&S->done)) return;
  KahanF mu, sg, ga;
  const float* __restrict__ p = W.p;
  const float* __restrict__ rt = Pc::on ? W.rt : W.r;
  auto gather = [&](int j) { return __ldg(p + j); };
  auto sums = [&](float sn, float pi, float rti, float dd) {
    mu.add(pi * sn);
    sg.add(rti * sn);
    ga.add((Pc::on ? dd * sn : sn) * sn);
  };
  // four rows per thread: the rows' own p, r~ and s move with 16-byte accesses
  const int n = op.n, nq = n >> 2;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nq; j += gridDim.x * blockDim.x) {
    const int i = 4 * j;
    const float4 s4 = rows32x4(op, i, p);
    *reinterpret_cast<float4*>(W.s + i) = s4;
    const float4 p4 = __ldg(reinterpret_cast<const float4*>(p + i));
    const float4 rt4 = __ldg(reinterpret_cast<const float4*>(rt + i));
    const float4 c4 = pc_quad32(pc, i);
    sums(s4.x, p4.x, rt4.x, c4.x);
    sums(s4.y, p4.y, rt4.y, c4.y);
    sums(s4.z, p4.z, rt4.z, c4.z);
    sums(s4.w, p4.w, rt4.w, c4.w);
  }
  if (blockIdx.x == gridDim.x - 1 && (int)threadIdx.x < n - 4 * nq) {
    const int i = 4 * nq + threadIdx.x;
    const float sn = op.row32(i, gather);
    W.s[i] = sn;
    sums(sn, __ldg(p + i), __ldg(rt + i), Pc::on ? (float)pc(i) : 1.f);
  }
  double acc[3] = {mu.value(), sg.value(), ga.value()};
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
    const int k = S->k + 1;
    S->mu = tot[0];
    S->sigma = tot[1];
    S->gamma = tot[2];
    S->nu = a2[0];
    S->rho = a2[1];
    if (!record_and_test(S, k, a2[1])) scalar_step_pr(S, false);
  }
}

// x += scale * d (FP64 refinement update).
template <class Op, class Pc>
__global__ void __launch_bounds__(kBlock) k_mx_update(Op op, Vecs V, Vecs32 W, double scale) {
  PRCG_ROWS(i, op.n) { V.x[i] = fma(scale, (double)W.d[i], V.x[i]); }
}

}  // namespace prcg
