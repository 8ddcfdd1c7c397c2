// Operators (y_i = sum_j a_ij g(j)) and Jacobi preconditioners.
//
// Every fused sweep evaluates the matrix-vector product of a vector that is
// itself being updated in the same sweep (Algorithm 2: s_k = A p_k with
// p_k = r~_k + beta_k p_{k-1}).  The operators therefore take a gather
// functor g(j) that returns the *new* value at column j, computed from the
// previous iteration's vectors; the owner of row j computes the identical
// expression, so the product uses exactly the stored p_k.
#pragma once

#include "prcg_common.cuh"
#include "prcg_isum.cuh"

namespace prcg {

enum OpKind { OP_CSR = 0, OP_ST2 = 1, OP_ST3 = 2, OP_VC2 = 3, OP_VC3 = 4, OP_SELL = 5, OP_DENSE = 6 };
enum PcKind { PC_NONE = 0, PC_SCALAR = 1, PC_VEC = 2 };

// Host-side description of an operator; the device structs below are built
// from it.
struct OpDesc {
  int kind;
  int n;
  int nx, ny, nz;
  const int* rp;
  const int* ci;
  const double* va;
  const double* fx;
  const double* fy;
  const double* fz;
  const double* adiag;   // variable-coefficient diagonal incl. shift
  double cdiag;          // constant-coefficient diagonal 2*dim + shift
  int cint;              // cdiag when it is an integer in [1, 8], else 0
  const int* sptr;       // SELL-32: first entry of each 32-row slice
  const int* slen;       // SELL-32: entries per row in each slice
  const int* scol;       // SELL-32 column indices, slice-major, row-minor
  const double* sval;    // SELL-32 values (padding: column = row, value 0)
  const float* sval32;   // FP32 copy of sval for the mixed-precision inner solve
  int tma;               // SELL-32 tiles fit the TMA stages: product sweeps stage entries in smem
  const double* da;      // dense: A column-major (= row-major, A symmetric), leading dimension lda
  int lda;               // dense: multiple of 32, >= n
  int ncb, cbw;          // dense: column blocks of the product and their width
  double* dpart[2];      // dense: partial products, [ncb][n] each
  FastDiv divx, divy;    // stencils: division by nx and by ny
};

struct PcDesc {
  int kind;
  const double* d;
  double dscalar;
};

// ---------------------------------------------------------------- CSR
struct CsrOp {
  const int* __restrict__ rp;
  const int* __restrict__ ci;
  const double* __restrict__ va;
  int n;
  explicit CsrOp(const OpDesc& o) : rp(o.rp), ci(o.ci), va(o.va), n(o.n) {}
  template <class G>
  __device__ __forceinline__ double row(int i, G&& g) const {
    const int e0 = __ldg(rp + i), e1 = __ldg(rp + i + 1);
    double acc = 0.0;
    for (int e = e0; e < e1; ++e) acc = fma(__ldg(va + e), g(__ldg(ci + e)), acc);
    return acc;
  }
  template <class G1, class G2>
  __device__ __forceinline__ void row2(int i, G1&& g1, G2&& g2, double& a1, double& a2) const {
    const int e0 = __ldg(rp + i), e1 = __ldg(rp + i + 1);
    double c1 = 0.0, c2 = 0.0;
    for (int e = e0; e < e1; ++e) {
      const double a = __ldg(va + e);
      const int j = __ldg(ci + e);
      c1 = fma(a, g1(j), c1);
      c2 = fma(a, g2(j), c2);
    }
    a1 = c1;
    a2 = c2;
  }
};

// ---------------------------------------------------------------- SELL-32
// The CSR matrix re-laid out in slices of 32 consecutive rows; entry t of
// row 32 s + l sits at sptr[s] + 32 t + l, so the 32 lanes of a warp (which
// own 32 consecutive rows) read each entry position with one coalesced
// access and run the same trip count.  Built from the caller's CSR at
// context creation; sums run in the same column order as the CSR rows.
struct SellOp {
  const int* __restrict__ sptr;
  const int* __restrict__ slen;
  const int* __restrict__ scol;
  const double* __restrict__ sval;
  int n;
  const float* __restrict__ sval32;
  explicit SellOp(const OpDesc& o)
      : sptr(o.sptr), slen(o.slen), scol(o.scol), sval(o.sval), n(o.n), sval32(o.sval32) {}
  // FP32 product row for the mixed-precision inner solve (FP32 values)
  template <class G>
  __device__ __forceinline__ float row32(int i, G&& g) const {
    const int sl = i >> 5;
    const int base = __ldg(sptr + sl) + (i & 31);
    const int L = __ldg(slen + sl);
    float acc = 0.f;
    for (int t = 0; t < L; ++t) acc = fmaf(__ldg(sval32 + base + 32 * t), g(__ldg(scol + base + 32 * t)), acc);
    return acc;
  }
  // Entries t < 8 are loaded with predication (all loads of a row are in
  // flight together); longer rows continue in a plain loop.
  template <class F>
  __device__ __forceinline__ void visit(int i, F&& f) const {
    const int sl = i >> 5;
    const int base = __ldg(sptr + sl) + (i & 31);
    const int L = __ldg(slen + sl);
    int j[8];
    double a[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const bool ok = t < L;
      j[t] = ok ? __ldg(scol + base + 32 * t) : i;
      a[t] = ok ? __ldg(sval + base + 32 * t) : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (t < L) f(j[t], a[t]);
    for (int t = 8; t < L; ++t) f(__ldg(scol + base + 32 * t), __ldg(sval + base + 32 * t));
  }
  // one FMA chain per row: the large sweeps are bound by FP64 issue, so a
  // second accumulator (one more FP64 add per row) would cost more than the
  // chain latency it hides
  template <class G>
  __device__ __forceinline__ double row(int i, G&& g) const {
    double acc = 0.0;
    visit(i, [&](int j, double a) { acc = fma(a, g(j), acc); });
    return acc;
  }
  template <class G1, class G2>
  __device__ __forceinline__ void row2(int i, G1&& g1, G2&& g2, double& a1, double& a2) const {
    double c1 = 0.0, c2 = 0.0;
    visit(i, [&](int j, double a) {
      c1 = fma(a, g1(j), c1);
      c2 = fma(a, g2(j), c2);
    });
    a1 = c1;
    a2 = c2;
  }
};

// ------------------------------------------- constant-coefficient stencil
// 5-point (DIM 2) / 7-point (DIM 3) Poisson with Dirichlet-0 boundary:
// y_i = cdiag * g(i) - sum over existing neighbours g(j).  The neighbour sum
// is exact in fixed point (prcg_isum.cuh) and rounded once, so the FP64 pipe
// -- the bottleneck of these sweeps on GB300 -- does one FMA per row instead
// of 2*DIM+1; the result differs from a sequential FP64 evaluation only in
// rounding (it is the more accurate of the two).
template <int DIM>
struct StencilOp {
  int nx, ny, nz, n;
  double cdiag;
  int cint;
  FastDiv divx, divy;
  explicit StencilOp(const OpDesc& o)
      : nx(o.nx), ny(o.ny), nz(o.nz), n(o.n), cdiag(o.cdiag), cint(o.cint), divx(o.divx),
        divy(o.divy) {}
  __device__ __forceinline__ void coords(int i, int& x, int& y, int& z) const {
    const int yz = fast_div(divx, i);
    x = i - yz * nx;
    z = DIM == 3 ? fast_div(divy, yz) : 0;
    y = yz - z * ny;
  }
  // ||A||_inf = max_i sum_j |a_ij| <= |cdiag| + 2*DIM
  __device__ __forceinline__ double anorm_inf() const { return fabs(cdiag) + 2.0 * DIM; }
  // f(j, coefficient) for the 2*DIM+1 entries in increasing column order.
  // Missing neighbours (Dirichlet boundary) are visited as column i with
  // coefficient 0, so every load is issued unconditionally.
  template <class F>
  __device__ __forceinline__ void visit(int i, F&& f) const {
    int x, y, z;
    coords(i, x, y, z);
    const int pl = nx * ny;
    if (DIM == 3) f(z > 0 ? i - pl : i, z > 0 ? -1.0 : 0.0);
    f(y > 0 ? i - nx : i, y > 0 ? -1.0 : 0.0);
    f(x > 0 ? i - 1 : i, x > 0 ? -1.0 : 0.0);
    f(i, cdiag);
    f(x < nx - 1 ? i + 1 : i, x < nx - 1 ? -1.0 : 0.0);
    f(y < ny - 1 ? i + nx : i, y < ny - 1 ? -1.0 : 0.0);
    if (DIM == 3) f(z < nz - 1 ? i + pl : i, z < nz - 1 ? -1.0 : 0.0);
  }
  // The 2*DIM neighbour values of row i (0 for a missing neighbour), every
  // load issued unconditionally.
  template <class G>
  __device__ __forceinline__ void neighbours(int i, int x, int y, int z, G&& g,
                                             double (&v)[2 * DIM]) const {
    const int pl = nx * ny;
    int t = 0;
    if (DIM == 3) {
      const double a = g(z > 0 ? i - pl : i);
      v[t++] = z > 0 ? a : 0.0;
    }
    {
      const double a = g(y > 0 ? i - nx : i);
      v[t++] = y > 0 ? a : 0.0;
    }
    {
      const double a = g(x > 0 ? i - 1 : i);
      v[t++] = x > 0 ? a : 0.0;
    }
    {
      const double a = g(x < nx - 1 ? i + 1 : i);
      v[t++] = x < nx - 1 ? a : 0.0;
    }
    {
      const double a = g(y < ny - 1 ? i + nx : i);
      v[t++] = y < ny - 1 ? a : 0.0;
    }
    if (DIM == 3) {
      const double a = g(z < nz - 1 ? i + pl : i);
      v[t++] = z < nz - 1 ? a : 0.0;
    }
  }
  // s_i = c p_i - sum of the neighbours: the sum on the integer pipes
  // (exact, rounded once), one FP64 FMA per row
  template <class G>
  __device__ __forceinline__ double row(int i, G&& g) const {
    int x, y, z;
    coords(i, x, y, z);
    double v[2 * DIM];
    neighbours(i, x, y, z, g, v);
    return fma(cdiag, g(i), -neighbour_sum<2 * DIM>(v));
  }
  // s_i = c p_i - sum of the neighbours, the sum taken from the block
  // fixed-point copy P of p (scale S, prcg_isum.cuh): 2*DIM 64-bit integer
  // adds and one exactly rounded conversion, then the one FP64 FMA.  With
  // kInt (c an integer in [1, 8], cint) the row's own term is taken from P
  // too: c P_i - sum P_j is exact in 64 bits (|.| < 14 * 2^58) and the row
  // is one exactly rounded conversion of it, no FP64 instruction; its error
  // is that of the copy, at most (c + 2*DIM) 2^-(S+1), normwise like the
  // neighbour sum's.
  template <bool kInt = false>
  __device__ __forceinline__ double row_fixed(int i, double pi, const long long* __restrict__ P,
                                              int S) const {
    int x, y, z;
    coords(i, x, y, z);
    const int pl = nx * ny;
    long long acc = 0;
    auto nb = [&](bool ok, int j) {
      const long long v = __ldg(P + (ok ? j : i));
      acc += ok ? v : 0ll;
    };
    if (DIM == 3) nb(z > 0, i - pl);
    nb(y > 0, i - nx);
    nb(x > 0, i - 1);
    nb(x < nx - 1, i + 1);
    nb(y < ny - 1, i + nx);
    if (DIM == 3) nb(z < nz - 1, i + pl);
    if constexpr (kInt) return fixed_to_double((long long)cint * __ldg(P + i) - acc, S);
    return fma(cdiag, pi, -fixed_to_double(acc, S));
  }
  // Rows i and i + 1 of one x-line (i even, nx even; g2(j) loads the pair
  // j, j + 1 for even j): the pair's own values and its y and z neighbours
  // with 16-byte loads, the two outer x neighbours alone.  Each row's terms
  // are neighbours()'s, in its order, so the results equal row()'s bit for
  // bit.
  __device__ __forceinline__ bool pairs_ok() const { return (nx & 1) == 0; }
  template <class G, class G2>
  __device__ __forceinline__ double2 rows2(int i, G&& g, G2&& g2) const {
    int x, y, z;
    coords(i, x, y, z);
    const int pl = nx * ny;
    const double2 c = g2(i);
    const double xl = g(x > 0 ? i - 1 : i), xr = g(x + 2 < nx ? i + 2 : i);
    const double2 ym = g2(y > 0 ? i - nx : i), yp = g2(y < ny - 1 ? i + nx : i);
    double2 zm = c, zp = c;
    if (DIM == 3) {
      zm = g2(z > 0 ? i - pl : i);
      zp = g2(z < nz - 1 ? i + pl : i);
    }
    double v0[2 * DIM], v1[2 * DIM];
    int t = 0;
    if (DIM == 3) {
      v0[t] = z > 0 ? zm.x : 0.0;
      v1[t++] = z > 0 ? zm.y : 0.0;
    }
    v0[t] = y > 0 ? ym.x : 0.0;
    v1[t++] = y > 0 ? ym.y : 0.0;
    v0[t] = x > 0 ? xl : 0.0;
    v1[t++] = c.x;
    v0[t] = c.y;
    v1[t++] = x + 2 < nx ? xr : 0.0;
    v0[t] = y < ny - 1 ? yp.x : 0.0;
    v1[t++] = y < ny - 1 ? yp.y : 0.0;
    if (DIM == 3) {
      v0[t] = z < nz - 1 ? zp.x : 0.0;
      v1[t++] = z < nz - 1 ? zp.y : 0.0;
    }
    return make_double2(fma(cdiag, c.x, -neighbour_sum<2 * DIM>(v0)),
                        fma(cdiag, c.y, -neighbour_sum<2 * DIM>(v1)));
  }
  // Rows i and i + 1 of one x-line (i even, nx even) from P: their x
  // neighbours inside the pair come from one 16-byte load of P[i], P[i+1],
  // the y and z neighbours from 16-byte loads of the neighbouring pairs.
  // The integer sums are exact, so each row equals row_fixed<kInt>'s bit
  // for bit.
  template <bool kInt = false>
  __device__ __forceinline__ double2 rows2_fixed(int i, double2 pi, const long long* __restrict__ P,
                                                 int S) const {
    int x, y, z;
    coords(i, x, y, z);
    const int pl = nx * ny;
    auto ld2 = [&](bool ok, int j) {
      const longlong2 v = __ldg(reinterpret_cast<const longlong2*>(P + (ok ? j : i)));
      return ok ? v : make_longlong2(0ll, 0ll);
    };
    const longlong2 c = __ldg(reinterpret_cast<const longlong2*>(P + i));
    long long a0 = c.y, a1 = c.x;   // row i: P[i+1]; row i+1: P[i]
    const long long xl = __ldg(P + (x > 0 ? i - 1 : i));
    const long long xr = __ldg(P + (x + 2 < nx ? i + 2 : i));
    a0 += x > 0 ? xl : 0ll;
    a1 += x + 2 < nx ? xr : 0ll;
    const longlong2 ym = ld2(y > 0, i - nx), yp = ld2(y < ny - 1, i + nx);
    a0 += ym.x + yp.x;
    a1 += ym.y + yp.y;
    if (DIM == 3) {
      const longlong2 zm = ld2(z > 0, i - pl), zp = ld2(z < nz - 1, i + pl);
      a0 += zm.x + zp.x;
      a1 += zm.y + zp.y;
    }
    if constexpr (kInt)
      return make_double2(fixed_to_double((long long)cint * c.x - a0, S),
                          fixed_to_double((long long)cint * c.y - a1, S));
    return make_double2(fma(cdiag, pi.x, -fixed_to_double(a0, S)),
                        fma(cdiag, pi.y, -fixed_to_double(a1, S)));
  }
  template <class G>
  __device__ __forceinline__ float row32(int i, G&& g) const {
    float acc = 0.f;
    visit(i, [&](int j, double a) { acc = fmaf((float)a, g(j), acc); });
    return acc;
  }
  template <class G1, class G2>
  __device__ __forceinline__ void row2(int i, G1&& g1, G2&& g2, double& a1, double& a2) const {
    int x, y, z;
    coords(i, x, y, z);
    double v[2 * DIM];
    neighbours(i, x, y, z, g1, v);
    a1 = fma(cdiag, g1(i), -neighbour_sum<2 * DIM>(v));
    neighbours(i, x, y, z, g2, v);
    a2 = fma(cdiag, g2(i), -neighbour_sum<2 * DIM>(v));
  }
};

// Operators whose product sweeps can read the block fixed-point copy of p.
template <class Op>
struct HasFixedRow : std::false_type {};
template <int DIM>
struct HasFixedRow<StencilOp<DIM>> : std::true_type {};

// Operators with a two-row product (rows2: rows i, i + 1 of one grid line).
template <class Op>
struct HasRows2 : std::false_type {};
template <int DIM>
struct HasRows2<StencilOp<DIM>> : std::true_type {};

// ------------------------------------------- variable-coefficient stencil
// A = sum_f c_f (e_a - e_b)(e_a - e_b)^T (+ shift I); diagonal precomputed.

// -c where `keep`, else +0.0, formed on the two 32-bit halves of c with
// integer operations.  Formed on the 64-bit value (a negated selection, or
// a 64-bit mask of the bits) it cost one FP64 instruction per coefficient
// on this GPU -- measured 12 FP64 instructions per face-stencil row instead
// of the 7 FMAs, and 40 % more time for the product.
__device__ __forceinline__ double neg_or_zero(bool keep, double c) {
  const unsigned m = keep ? 0xFFFFFFFFu : 0u;
  return __hiloint2double((int)(((unsigned)__double2hiint(c) ^ 0x80000000u) & m),
                          (int)((unsigned)__double2loint(c) & m));
}

template <int DIM>
struct VarStencilOp {
  int nx, ny, nz, n;
  const double* __restrict__ fx;
  const double* __restrict__ fy;
  const double* __restrict__ fz;
  const double* __restrict__ adiag;
  FastDiv divx, divy;
  explicit VarStencilOp(const OpDesc& o)
      : nx(o.nx), ny(o.ny), nz(o.nz), n(o.n), fx(o.fx), fy(o.fy), fz(o.fz), adiag(o.adiag),
        divx(o.divx), divy(o.divy) {}
  template <class F>
  __device__ __forceinline__ void visit(int i, F&& f) const {
    const int yz = fast_div(divx, i);
    const int x = i - yz * nx;
    const int z = DIM == 3 ? fast_div(divy, yz) : 0;
    const int y = yz - z * ny;
    const int pl = nx * ny;
    // face coefficients of the cell (boundary faces are valid addresses)
    const double czm = DIM == 3 ? __ldg(fz + i) : 0.0;
    const double cym = __ldg(fy + (z * (ny + 1) + y) * nx + x);
    const double cxm = __ldg(fx + yz * (nx + 1) + x);
    const double cxp = __ldg(fx + yz * (nx + 1) + x + 1);
    const double cyp = __ldg(fy + (z * (ny + 1) + y + 1) * nx + x);
    const double czp = DIM == 3 ? __ldg(fz + i + pl) : 0.0;
    // off-diagonal coefficients -c_f, zero for a missing neighbour, formed on
    // the integer pipes
    if (DIM == 3) f(z > 0 ? i - pl : i, neg_or_zero(z > 0, czm));
    f(y > 0 ? i - nx : i, neg_or_zero(y > 0, cym));
    f(x > 0 ? i - 1 : i, neg_or_zero(x > 0, cxm));
    f(i, __ldg(adiag + i));
    f(x < nx - 1 ? i + 1 : i, neg_or_zero(x < nx - 1, cxp));
    f(y < ny - 1 ? i + nx : i, neg_or_zero(y < ny - 1, cyp));
    if (DIM == 3) f(z < nz - 1 ? i + pl : i, neg_or_zero(z < nz - 1, czp));
  }
  // one FMA chain per row: the large sweeps are bound by FP64 issue, so a
  // second accumulator (one more FP64 add per row) would cost more than the
  // chain latency it hides
  template <class G>
  __device__ __forceinline__ double row(int i, G&& g) const {
    double acc = 0.0;
    visit(i, [&](int j, double a) { acc = fma(a, g(j), acc); });
    return acc;
  }
  // Rows i and i + 1 of one x-line (i even, nx even; the face arrays and the
  // diagonal start on 16-byte boundaries; g2(j) loads the pair j, j + 1 for
  // even j).  The x-face between the two rows is read once; the y- and
  // z-faces, the diagonals, the pair's own values and its y and z
  // neighbours come in 16-byte loads -- 16 load instructions for two rows
  // instead of 30.  Each row's FMA chain is visit()'s (missing neighbours
  // as coefficient 0 times the row's own value, the same order), so the
  // results equal row()'s bit for bit.
  __device__ __forceinline__ bool pairs_ok() const { return (nx & 1) == 0; }
  template <class G, class G2>
  __device__ __forceinline__ double2 rows2(int i, G&& g, G2&& g2) const {
    const int yz = fast_div(divx, i);
    const int x = i - yz * nx;
    const int z = DIM == 3 ? fast_div(divy, yz) : 0;
    const int y = yz - z * ny;
    const int pl = nx * ny;
    auto ld2 = [](const double* q) { return __ldg(reinterpret_cast<const double2*>(q)); };
    const double* fxr = fx + yz * (nx + 1) + x;
    const double cx0 = __ldg(fxr), cx1 = __ldg(fxr + 1), cx2 = __ldg(fxr + 2);
    const double2 cym = ld2(fy + (z * (ny + 1) + y) * nx + x);
    const double2 cyp = ld2(fy + (z * (ny + 1) + y + 1) * nx + x);
    double2 czm = make_double2(0.0, 0.0), czp = czm;
    if (DIM == 3) {
      czm = ld2(fz + i);
      czp = ld2(fz + i + pl);
    }
    const double2 dg = ld2(adiag + i);
    const double2 c = g2(i);
    const double xl = g(x > 0 ? i - 1 : i), xr = g(x + 2 < nx ? i + 2 : i + 1);
    const double2 ym = g2(y > 0 ? i - nx : i), yp = g2(y < ny - 1 ? i + nx : i);
    double2 zm = c, zp = c;
    if (DIM == 3) {
      zm = g2(z > 0 ? i - pl : i);
      zp = g2(z < nz - 1 ? i + pl : i);
    }
    // a missing neighbour is loaded from the row itself (the clamped index)
    // with its coefficient masked to zero, as in visit
    const double ncx1 = neg_or_zero(true, cx1);
    double a0 = 0.0, a1 = 0.0;
    if (DIM == 3) {
      a0 = fma(neg_or_zero(z > 0, czm.x), zm.x, a0);
      a1 = fma(neg_or_zero(z > 0, czm.y), zm.y, a1);
    }
    a0 = fma(neg_or_zero(y > 0, cym.x), ym.x, a0);
    a1 = fma(neg_or_zero(y > 0, cym.y), ym.y, a1);
    a0 = fma(neg_or_zero(x > 0, cx0), xl, a0);
    a1 = fma(ncx1, c.x, a1);
    a0 = fma(dg.x, c.x, a0);
    a1 = fma(dg.y, c.y, a1);
    a0 = fma(ncx1, c.y, a0);
    a1 = fma(neg_or_zero(x + 2 < nx, cx2), xr, a1);
    a0 = fma(neg_or_zero(y < ny - 1, cyp.x), yp.x, a0);
    a1 = fma(neg_or_zero(y < ny - 1, cyp.y), yp.y, a1);
    if (DIM == 3) {
      a0 = fma(neg_or_zero(z < nz - 1, czp.x), zp.x, a0);
      a1 = fma(neg_or_zero(z < nz - 1, czp.y), zp.y, a1);
    }
    return make_double2(a0, a1);
  }
  template <class G>
  __device__ __forceinline__ float row32(int i, G&& g) const {
    float acc = 0.f;
    visit(i, [&](int j, double a) { acc = fmaf((float)a, g(j), acc); });
    return acc;
  }
  template <class G1, class G2>
  __device__ __forceinline__ void row2(int i, G1&& g1, G2&& g2, double& a1, double& a2) const {
    double c1 = 0.0, c2 = 0.0;
    visit(i, [&](int j, double a) {
      c1 = fma(a, g1(j), c1);
      c2 = fma(a, g2(j), c2);
    });
    a1 = c1;
    a2 = c2;
  }
};

template <int DIM>
struct HasRows2<VarStencilOp<DIM>> : std::true_type {};

// ------------------------------------------------------------ dense matrix
// Symmetric dense A (the paper's Section 5 model problem, stored dense to
// make the two products of pipe-PR-CG cost a full pass over A).  A product
// y = A v is formed before the sweep that needs it by dense_units()
// (prcg_dense.cuh): warp units of 32 rows x one column block write partial
// sums part[c][i]; row(i, .) then adds the ncb partials of row i in column
// block order, so the result does not depend on the launch shape.  The
// gather argument of row() is ignored -- the caller has already formed the
// product of the vector that gather would read.
constexpr int kMaxDenseN = 1 << 17;        // A of up to 137 GB
constexpr int kDensePersistMax = 4096;     // dense solves up to this n run persistent

struct DenseOp {
  int n, lda, ncb, cbw;
  const double* __restrict__ A;
  double* part0;
  double* part1;
  explicit DenseOp(const OpDesc& o)
      : n(o.n), lda(o.lda), ncb(o.ncb), cbw(o.cbw), A(o.da), part0(o.dpart[0]), part1(o.dpart[1]) {}
  __device__ __forceinline__ double sum_parts(const double* part, int i) const {
    double acc = __ldcg(part + i);
    for (int c = 1; c < ncb; ++c) acc += __ldcg(part + (size_t)c * n + i);
    return acc;
  }
  template <class G>
  __device__ __forceinline__ double row(int i, G&&) const {
    return sum_parts(part0, i);
  }
  template <class G1, class G2>
  __device__ __forceinline__ void row2(int i, G1&&, G2&&, double& a1, double& a2) const {
    a1 = sum_parts(part0, i);
    a2 = sum_parts(part1, i);
  }
};

// The preconditioner's d_i, d_{i+1} (i even; vectors start on 256-byte
// boundaries, so the pair is one 16-byte load for a Jacobi vector).
template <class Pc>
__device__ __forceinline__ double2 pc_pair(const Pc& pc, int i) {
  return make_double2(pc(i), pc(i + 1));
}

template <class Op>
struct IsDense : std::false_type {};
template <>
struct IsDense<DenseOp> : std::true_type {};

// ------------------------------------------------------ preconditioners
struct PcNone {
  static constexpr bool on = false;
  explicit PcNone(const PcDesc&) {}
  __device__ __forceinline__ double operator()(int) const { return 1.0; }
};
struct PcScalar {
  static constexpr bool on = true;
  double d;
  explicit PcScalar(const PcDesc& p) : d(p.dscalar) {}
  __device__ __forceinline__ double operator()(int) const { return d; }
};
struct PcVec {
  static constexpr bool on = true;
  const double* __restrict__ d;
  explicit PcVec(const PcDesc& p) : d(p.d) {}
  __device__ __forceinline__ double operator()(int i) const { return __ldg(d + i); }
};

__device__ __forceinline__ double2 pc_pair(const PcVec& pc, int i) {
  return __ldg(reinterpret_cast<const double2*>(pc.d + i));
}

}  // namespace prcg
