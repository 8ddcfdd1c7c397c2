// Host harness for tests/test_isum_host_cpu.py: runs the stencil kernels'
// integer-pipe helpers (csrc/prcg_isum.cuh) on the CPU.
//
//   isum_host_check sum <in> <out>   in: int32 K, int64 count, count*K doubles;
//                                    out: count doubles (the neighbour sum) and
//                                    count int8 flags (1: fixed point taken)
//   isum_host_check fx <in> <out>    in: int32 K, int64 count, int32 S, count*K
//                                    doubles; out: count doubles (the sum of the
//                                    K block-fixed-point values P_j = round(v_j 2^S),
//                                    converted back), count int64 (that integer
//                                    sum) and count int8 flags (1: a value did
//                                    not fit the window)
//   isum_host_check scale <in> <out> in: int64 count, count doubles B; out: count
//                                    int32 fixed_scale(B) and count doubles
//                                    amax_bound(high word of |B|)
//   isum_host_check div <d> <n>      floor(v / d) through the invariant-divisor
//                                    quotient for v in [0, n) (n <= 2^31 - 1): every
//                                    v of the lowest and highest 2^22 values and
//                                    k*d - 1, k*d, k*d + 1 for up to 2^22 values
//                                    of k spread over the range; prints the number
//                                    of mismatches and of values checked
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../paper_1905_01549_gb300/csrc/prcg_isum.cuh"

template <int K>
static void run_sum(const std::vector<double>& v, int64_t count, std::vector<double>& out,
                    std::vector<int8_t>& fixed) {
  for (int64_t t = 0; t < count; ++t) {
    double a[K];
    for (int j = 0; j < K; ++j) a[j] = v[t * K + j];
    double s = 0.0;
    fixed[t] = prcg::fixed_point_sum<K>(a, s) ? 1 : 0;
    if (!fixed[t]) {
      s = a[0];
      for (int j = 1; j < K; ++j) s += a[j];
    }
    out[t] = s;
  }
}

int main(int argc, char** argv) {
  if (argc == 4 && !std::strcmp(argv[1], "sum")) {
    FILE* f = std::fopen(argv[2], "rb");
    if (!f) return 2;
    int32_t K = 0;
    int64_t count = 0;
    if (std::fread(&K, 4, 1, f) != 1 || std::fread(&count, 8, 1, f) != 1 || count < 0) return 3;
    std::vector<double> v((size_t)count * K);
    if (count && std::fread(v.data(), 8, v.size(), f) != v.size()) return 4;
    std::fclose(f);
    std::vector<double> out((size_t)count);
    std::vector<int8_t> fixed((size_t)count);
    if (K == 4)
      run_sum<4>(v, count, out, fixed);
    else if (K == 6)
      run_sum<6>(v, count, out, fixed);
    else
      return 5;
    FILE* g = std::fopen(argv[3], "wb");
    if (!g) return 6;
    std::fwrite(out.data(), 8, out.size(), g);
    std::fwrite(fixed.data(), 1, fixed.size(), g);
    std::fclose(g);
    return 0;
  }
  if (argc == 4 && !std::strcmp(argv[1], "fx")) {
    FILE* f = std::fopen(argv[2], "rb");
    if (!f) return 2;
    int32_t K = 0, S = 0;
    int64_t count = 0;
    if (std::fread(&K, 4, 1, f) != 1 || std::fread(&count, 8, 1, f) != 1 ||
        std::fread(&S, 4, 1, f) != 1 || count < 0 || K < 1 || K > 8)
      return 3;
    std::vector<double> v((size_t)count * K);
    if (count && std::fread(v.data(), 8, v.size(), f) != v.size()) return 4;
    std::fclose(f);
    std::vector<double> out((size_t)count);
    std::vector<int64_t> sums((size_t)count);
    std::vector<int8_t> bad((size_t)count);
    for (int64_t t = 0; t < count; ++t) {
      bool b = false;
      long long acc = 0;
      for (int j = 0; j < K; ++j) acc += prcg::to_fixed(v[t * K + j], S, b);
      sums[t] = acc;
      bad[t] = b ? 1 : 0;
      out[t] = b ? 0.0 : prcg::fixed_to_double(acc, S);
    }
    FILE* g = std::fopen(argv[3], "wb");
    if (!g) return 6;
    std::fwrite(out.data(), 8, out.size(), g);
    std::fwrite(sums.data(), 8, sums.size(), g);
    std::fwrite(bad.data(), 1, bad.size(), g);
    std::fclose(g);
    return 0;
  }
  if (argc == 4 && !std::strcmp(argv[1], "scale")) {
    FILE* f = std::fopen(argv[2], "rb");
    if (!f) return 2;
    int64_t count = 0;
    if (std::fread(&count, 8, 1, f) != 1 || count < 0) return 3;
    std::vector<double> v((size_t)count);
    if (count && std::fread(v.data(), 8, v.size(), f) != v.size()) return 4;
    std::fclose(f);
    std::vector<int32_t> sc((size_t)count);
    std::vector<double> bd((size_t)count);
    for (int64_t t = 0; t < count; ++t) {
      sc[t] = prcg::fixed_scale(v[t]);
      bd[t] = prcg::amax_bound(prcg::isum_hi(v[t]) & 0x7FFFFFFFu);
    }
    FILE* g = std::fopen(argv[3], "wb");
    if (!g) return 6;
    std::fwrite(sc.data(), 4, sc.size(), g);
    std::fwrite(bd.data(), 8, bd.size(), g);
    std::fclose(g);
    return 0;
  }
  if (argc == 4 && !std::strcmp(argv[1], "div")) {
    const int d = std::atoi(argv[2]);
    const long long n = std::atoll(argv[3]);
    if (d < 1 || n < 0 || n > 2147483647LL) return 7;
    const prcg::FastDiv fd = prcg::make_fastdiv(d);
    long long bad = 0, checked = 0;
    auto check = [&](long long v) {
      if (v < 0 || v >= n) return;
      ++checked;
      if (prcg::fast_div(fd, (int)v) != (int)(v / d)) ++bad;
    };
    const long long w = 1LL << 22;
    for (long long v = 0; v < w; ++v) check(v);
    for (long long v = n - w; v < n; ++v) check(v);
    const long long kmax = (n - 1) / d;
    const long long step = kmax / w + 1;
    for (long long k = 0; k <= kmax; k += step) {
      check(k * d - 1);
      check(k * d);
      check(k * d + 1);
    }
    std::printf("%lld %lld\n", bad, checked);
    return 0;
  }
  std::fprintf(stderr, "usage: isum_host_check sum <in> <out> | div <d> <n>\n");
  return 1;
}
