// Integer-pipe helpers for the constant-coefficient stencil product.
//
// A GB300 SM issues FP64 at 2 lanes per clock, 64x below its FP32 and 32x
// below its integer rate, so a 7-point stencil row costs 7 FP64 FMAs of
// issue while its memory traffic needs only a fraction of that time.  The
// neighbour sum of a constant-coefficient stencil needs no multiplication:
// it is formed here exactly in 64-bit fixed point on the integer pipes and
// rounded once, which leaves the FP64 pipe one FMA (c p_i - sum) per row
// (none where the row is taken from a block fixed-point copy of p with an
// integer c, see StencilOp::row_fixed).
#pragma once

#include <cstdint>
#include <cstring>

namespace prcg {

// Bit access used by the fixed-point sum, on the device through intrinsics
// and on the host (tests) through memcpy and the compiler builtin.
__host__ __device__ __forceinline__ unsigned isum_hi(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(v);
#else
  uint64_t u;
  std::memcpy(&u, &v, 8);
  return (unsigned)(u >> 32);
#endif
}
__host__ __device__ __forceinline__ unsigned isum_lo(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(v);
#else
  uint64_t u;
  std::memcpy(&u, &v, 8);
  return (unsigned)u;
#endif
}
__host__ __device__ __forceinline__ double isum_from_bits(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double v;
  std::memcpy(&v, &u, 8);
  return v;
#endif
}
__host__ __device__ __forceinline__ int isum_clz64(uint64_t a) {   // a != 0
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return __builtin_clzll(a);
#endif
}

// Division by an invariant divisor d >= 1 (Granlund and Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Fig. 4.1):
// with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
//   q = (t + ((n - t) >> sh1)) >> sh2,  t = mulhi(m, n),
//   sh1 = min(l, 1), sh2 = max(l - 1, 0)
// equals floor(n / d) for every 32-bit unsigned n.  The stencil sweeps use
// it for the grid coordinates of a row: a division by a run-time divisor
// otherwise compiles to a long sequence that includes a slow-pipe
// reciprocal.
struct FastDiv {
  unsigned m;
  int sh1, sh2;
};

inline FastDiv make_fastdiv(int d) {
  int l = 0;
  while ((1ull << l) < (unsigned long long)d) ++l;
  FastDiv f;
  f.m = (unsigned)(((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d +
                   1ull);
  f.sh1 = l < 1 ? l : 1;
  f.sh2 = l > 1 ? l - 1 : 0;
  return f;
}

__host__ __device__ __forceinline__ unsigned mulhi32(unsigned a, unsigned b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (unsigned)(((unsigned long long)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ int fast_div(const FastDiv& f, int n) {
  const unsigned t = mulhi32(f.m, (unsigned)n);
  return (int)((t + (((unsigned)n - t) >> f.sh1)) >> f.sh2);
}

// Sum of K doubles in 64-bit fixed point.  Every term is placed in a window
// whose top is the largest exponent E among the terms: a term's 53-bit
// significand is shifted left by 7 (bit 59 for the largest terms, leaving
// headroom for the carries of up to 8 terms and the sign) and right by
// E - e_j, so bits more than 59 binades below the largest term are cut; the
// integer sum is then rounded once to nearest-even.  The result lies within
// one rounding of the exact sum plus K * 2^(E-1082) (the cut bits: at most
// K * 2^-59 times the largest term), tighter than K - 1 sequential FP64
// additions (their bound is about (K-1) eps times the sum of |terms|).
// Negation is done as a one's complement with the +1 of every negative term
// added once at the end.
//
// Returns false, leaving out untouched, when a term is infinite or NaN
// (E = 2047), when the result could overflow (E > 2040), or when every term
// is below 2^-959 (E < 64, which includes all-zero input): the caller adds
// those natively.  Zero and subnormal terms next to a term with E >= 64 lie
// at least 64 binades below the window and contribute nothing, which is
// within the stated bound.
template <int K>
__host__ __device__ __forceinline__ bool fixed_point_sum(const double (&v)[K], double& out) {
  unsigned hi[K], lo[K];
  unsigned mx = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    hi[j] = isum_hi(v[j]);
    lo[j] = isum_lo(v[j]);
    const unsigned mag = hi[j] & 0x7FFFFFFFu;
    mx = mag > mx ? mag : mx;
  }
  const int E = (int)(mx >> 20);
  if (E < 64 || E > 2040) return false;
  long long acc = 0;
  int neg = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const unsigned sg = (unsigned)((int)hi[j] >> 31);   // all ones for a negative term
    const unsigned mh = (hi[j] & 0xFFFFFu) | 0x100000u;
    const uint64_t m = ((uint64_t)mh << 39) | ((uint64_t)lo[j] << 7);
    // a significand shifted by 63 is 0, so the shift is clamped there
    const int dd = E - (int)((hi[j] >> 20) & 0x7FFu);
    const int d = dd < 63 ? dd : 63;
    acc += (long long)((m >> d) ^ (((uint64_t)sg << 32) | sg));
    neg -= (int)sg;
  }
  acc += neg;
  if (acc == 0) {
    out = 0.0;
    return true;
  }
  // |acc| < 2^63; the value is acc * 2^(E - 1082)
  const long long sm = acc >> 63;
  uint64_t a = (uint64_t)((acc ^ sm) - sm);
  const int lz = isum_clz64(a);
  a <<= lz;
  uint64_t mant = a >> 11;   // 53 bits, the leading one at bit 52
  const unsigned rem = (unsigned)a & 0x7FFu;
  mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  // biased exponent E + 4 - lz; adding the significand (leading one
  // included) to (exponent - 1) << 52 also carries a rounding overflow
  const uint64_t bits = ((uint64_t)(E + 3 - lz) << 52) + mant;
  out = isum_from_bits(bits | ((uint64_t)sm << 63));
  return true;
}

// ---------------------------------------------------------------------------
// Block fixed point with one scale per vector.
//
// The sweep that forms p also stores P_i = round(p_i 2^S) as a 64-bit
// integer, with one scale S for the whole vector, chosen before the sweep
// from an upper bound B >= max |p_i| so that B 2^S < 2^58 (to_fixed flags a
// value that does not fit).  The product sweep then adds the 2*dim
// neighbour values P_j with 64-bit integer adds and converts the sum once,
// exactly rounded, to FP64 (fixed_to_double).  The sum of the P_j is exact;
// the only errors are the roundings of the P_j (at most 2^-(S+1) each, i.e.
// 2^-59 B per term) and the one final rounding -- a normwise bound (relative
// to B, not to the row's own terms) far below the FP64 product's
// eps ||A|| ||p||.

// round(v 2^S) for |v| 2^S < 2^58 (half-way cases away from zero).  Zero,
// subnormal v and values below half a unit give 0; a value too large for
// the window, an infinity or a NaN sets bad.
__host__ __device__ __forceinline__ long long to_fixed(double v, int S, bool& bad) {
  const unsigned hi = isum_hi(v), lo = isum_lo(v);
  const int e = (int)((hi >> 20) & 0x7FFu);
  if (e == 0) return 0;
  // the significand m (53 bits) shifted up by 5: v 2^S = (m << 5) 2^(e - 1080 + S)
  const int t = 1080 - S - e;
  if (e == 0x7FF || t < 0) {
    bad = true;
    return 0;
  }
  if (t > 63) return 0;
  const uint64_t m = ((((uint64_t)((hi & 0xFFFFFu) | 0x100000u)) << 32) | lo) << 5;
  // m / 2^t rounded half away from zero (t == 0: exact)
  const uint64_t q = t == 0 ? m : ((m >> (t - 1)) + 1) >> 1;
  return (hi >> 31) ? -(long long)q : (long long)q;
}

// acc 2^-S as the nearest double (ties to even); |acc| < 2^63, and the
// scale keeps the result a normal number (|S| <= 900).
__host__ __device__ __forceinline__ double fixed_to_double(long long acc, int S) {
  if (acc == 0) return 0.0;
  const long long sm = acc >> 63;
  uint64_t a = (uint64_t)((acc ^ sm) - sm);
  const int lz = isum_clz64(a);
  a <<= lz;
  uint64_t mant = a >> 11;   // 53 bits, the leading one at bit 52
  const unsigned rem = (unsigned)a & 0x7FFu;
  mant += (rem > 0x400u || (rem == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  // value = a 2^-(lz + S) with a's leading one at bit 63: biased exponent
  // 1023 + 63 - lz - S; adding the significand (leading one included) to
  // (exponent - 1) << 52 also carries a rounding overflow
  const uint64_t bits = ((uint64_t)(1085 - lz - S) << 52) + mant;
  return isum_from_bits(bits | ((uint64_t)sm << 63));
}

// Scale S of a vector whose entries are bounded by B: the largest S with
// B 2^S < 2^58, or kNoScale when B is zero, not finite or out of range.
constexpr int kNoScale = -100000;
__host__ __device__ __forceinline__ int fixed_scale(double B) {
  if (!(B > 0.0) || !(B < 1e300)) return kNoScale;
  const unsigned hi = isum_hi(B);
  const int e = (int)((hi >> 20) & 0x7FFu) - 1022;   // B < 2^e
  if (e < -900 || e > 900) return kNoScale;
  return 58 - e;
}

// Upper bound of the magnitudes whose high words (sign cleared) have the
// maximum `hiw`: the double with high word hiw + 1 (0 for hiw == 0).
__host__ __device__ __forceinline__ double amax_bound(unsigned hiw) {
  if (hiw == 0) return 0.0;
  return isum_from_bits((uint64_t)(hiw + 1u) << 32);
}

// The neighbour sum of a stencil row: fixed point where it applies,
// otherwise (non-finite or extreme terms) the plain FP64 sum, so that NaN
// and infinity propagate as in FP64 arithmetic.
template <int K>
__device__ __forceinline__ double neighbour_sum(const double (&v)[K]) {
  double s;
  if (!fixed_point_sum<K>(v, s)) {
    s = v[0];
#pragma unroll
    for (int j = 1; j < K; ++j) s += v[j];
  }
  return s;
}

}  // namespace prcg
