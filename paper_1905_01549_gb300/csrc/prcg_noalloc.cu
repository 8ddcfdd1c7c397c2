// prcg_pr_solve_stencil_noalloc: PR-CG on a small constant-coefficient
// stencil without any device allocation.
//
// Some callers cannot allocate device memory: code running inside another
// framework's memory pool or allocator hooks, real-time loops that forbid
// cudaMalloc/cudaFree after start-up (they can synchronise the device or
// fail under a pool limit), and callers that must not hold a library
// context.  For them this entry point runs the whole PR-CG solve as one
// single-CTA kernel -- the PR sweep of prcg_kernels.cuh with the grid-wide
// reduction replaced by a block reduction -- and keeps every iteration
// vector in a file-scope device array of fixed size.  The caller passes only
// b and x (device memory it owns).
//
// The scratch array is allocated by the CUDA module loader when the library
// is loaded and stays resident on every device that loads the library until
// the process exits: kNoallocMaxN * 8 vectors * 8 bytes = 4 MiB plus a
// small header.  Every call uses the same array, so calls that overlap on the
// GPU (two streams, or two host threads) race on it and corrupt each other;
// serialise them.  Each call rewrites all scratch it reads before reading it.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>

#include "../../include/prcg.h"
#include "prcg_reduce.cuh"

namespace {

constexpr int kNoallocMaxN = 65536;       // largest n the scratch holds
constexpr int kNoallocThreads = 1024;
constexpr int kNoallocVectors = 8;        // r, r~, p, s, each double-buffered
constexpr int kHeaderDoubles = 32;
// The solve is one kernel that cannot be interrupted; maxit is bounded so
// that a tolerance the system cannot reach ends in bounded time.
constexpr int64_t kNoallocMaxItPerRow = 4;
constexpr int64_t kNoallocMaxItExtra = 1000;
constexpr int kMaxDevices = 64;

// file-scope scratch: [header][8 vectors of kNoallocMaxN doubles]
static __device__ __align__(256) double g_noalloc_scratch[kHeaderDoubles +
                                                          kNoallocVectors * kNoallocMaxN];

// Device address of the scratch array per device, null until the first call
// on that device looks it up.  Several host threads may make their first
// call at once: each then stores the same address, which the symbol lookup
// returns for that device every time.
std::atomic<double*> g_scratch_ptr[kMaxDevices];

struct NoallocArgs {
  int dim, nx, ny, nz, n;
  double cdiag;     // 2 * dim + shift
  double d;         // Jacobi scalar 1 / cdiag, or 1 when unpreconditioned
  int jacobi;
  const double* b;
  double* x;
  double* hist;     // device or NULL
  double tol;
  int maxit;
};

__device__ __forceinline__ double apply_row(const NoallocArgs& a, int i, const double* __restrict__ v) {
  // y_i = cdiag v_i - sum of existing neighbours (7/5-point, Dirichlet-0)
  const int x = i % a.nx, yz = i / a.nx, y = yz % a.ny, z = yz / a.ny;
  const int pl = a.nx * a.ny;
  double acc = 0.0;
  if (a.dim == 3 && z > 0) acc = fma(-1.0, v[i - pl], acc);
  if (y > 0) acc = fma(-1.0, v[i - a.nx], acc);
  if (x > 0) acc = fma(-1.0, v[i - 1], acc);
  acc = fma(a.cdiag, v[i], acc);
  if (x < a.nx - 1) acc = fma(-1.0, v[i + 1], acc);
  if (y < a.ny - 1) acc = fma(-1.0, v[i + a.nx], acc);
  if (a.dim == 3 && z < a.nz - 1) acc = fma(-1.0, v[i + pl], acc);
  return acc;
}

// The whole PR-CG run (initialize(), then Algorithm 2 with the scalars
// formed at the start of each iteration) in one CTA.  Vectors live in the
// scratch array; they are written and read by different threads of this CTA
// between __syncthreads, so plain (coherent) loads are used throughout.
__global__ void __launch_bounds__(kNoallocThreads)
k_pr_noalloc(NoallocArgs a, double* scratch) {
  __shared__ double sm[5 * 32];
  __shared__ double sc[4];     // alpha, beta, continue flag
  double* hdr = scratch;
  const int n = a.n;
  double* V = scratch + kHeaderDoubles;
  double* r[2] = {V, V + kNoallocMaxN};
  double* rt[2] = {V + 2 * kNoallocMaxN, V + 3 * kNoallocMaxN};
  double* p[2] = {V + 4 * kNoallocMaxN, V + 5 * kNoallocMaxN};
  double* s[2] = {V + 6 * kNoallocMaxN, V + 7 * kNoallocMaxN};
  const int tid = threadIdx.x;
  const double d = a.d;
  // header state from a previous call is cleared first
  if (tid < kHeaderDoubles) hdr[tid] = 0.0;

  // initialize(): r_0 = b - A x_0, r~_0 = d r_0, p_0 = r~_0
  double acc3[3] = {0.0, 0.0, 0.0};
  for (int i = tid; i < n; i += kNoallocThreads) {
    const double ri = a.b[i] - apply_row(a, i, a.x);
    const double rti = a.jacobi ? d * ri : ri;
    r[0][i] = ri;
    rt[0][i] = rti;
    p[0][i] = rti;
    acc3[0] += rti * ri;
    acc3[1] += ri * ri;
    acc3[2] += a.b[i] * a.b[i];
  }
  prcg::block_sum<3>(acc3, sm);
  __shared__ double st_nu, st_bn2;
  if (tid == 0) {
    st_nu = acc3[0];
    st_bn2 = acc3[2];
    // b == 0 counts as converged; a non-finite ||b|| stays non-finite, so the
    // stopping test fails and the scalar step reports the breakdown
    double rel = acc3[2] != 0.0 ? sqrt(acc3[1]) / sqrt(acc3[2]) : 0.0;
    if (a.hist) a.hist[0] = rel;
    int status = -100;
    if (acc3[2] == 0.0 || rel <= a.tol) status = 0;
    else if (a.maxit == 0) status = 1;
    hdr[0] = status;
    hdr[1] = 0;                      // K
    hdr[2] = acc3[2] == 0.0 ? 1 : 0; // zero right-hand side
    sc[2] = status == -100 ? 1.0 : 0.0;
  }
  __syncthreads();
  // s_0 = A p_0; mu_0, sigma_0, gamma_0
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (sc[2] != 0.0) {
    for (int i = tid; i < n; i += kNoallocThreads) {
      const double si = apply_row(a, i, p[0]);
      s[0][i] = si;
      const double sti = a.jacobi ? d * si : si;
      acc[0] += p[0][i] * si;
      acc[1] += rt[0][i] * si;
      acc[2] += sti * si;
    }
  }
  prcg::block_sum<5>(acc, sm);
  double nu = 0.0, mu = 0.0, sigma = 0.0, gamma = 0.0;
  if (tid == 0) {
    nu = st_nu;
    mu = acc[0];
    sigma = acc[1];
    gamma = acc[2];
  }
  for (int k = 1; k <= a.maxit; ++k) {
    // scalar step: alpha_{k-1}, nu'_k (Eq. 2.3), beta_k
    if (tid == 0) {
      bool go = sc[2] != 0.0;
      if (go) {
        const double alpha = nu / mu;
        const double nu_pred = nu - 2.0 * alpha * sigma + alpha * alpha * gamma;
        if (!isfinite(nu) || !isfinite(mu) || !(mu > 0.0) || nu < 0.0 || !isfinite(nu_pred) ||
            nu_pred < 0.0 || nu == 0.0) {
          hdr[0] = 2;     // breakdown, K = k - 1
          go = false;
        } else {
          sc[0] = alpha;
          sc[1] = nu_pred / nu;
        }
      }
      sc[2] = go ? 1.0 : 0.0;
    }
    __syncthreads();
    if (sc[2] == 0.0) break;
    const double alpha = sc[0], beta = sc[1];
    const int qr = (k - 1) & 1, qw = k & 1;
    const double* pr_ = p[qr];
    const double* rr_ = r[qr];
    const double* rtr_ = rt[qr];
    const double* sr_ = s[qr];
    double a5[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = tid; i < n; i += kNoallocThreads) {
      // p_k at every column the row touches, from iteration k-1's vectors
      const int x = i % a.nx, yz = i / a.nx, y = yz % a.ny, z = yz / a.ny;
      const int pl = a.nx * a.ny;
      auto pnew = [&](int j) {
        const double sj = sr_[j];
        const double rtn = a.jacobi ? fma(-alpha, d * sj, rtr_[j]) : fma(-alpha, sj, rr_[j]);
        return fma(beta, pr_[j], rtn);
      };
      const double pi = pr_[i], si = sr_[i];
      a.x[i] = fma(alpha, pi, a.x[i]);
      const double rn = fma(-alpha, si, rr_[i]);
      const double rtn = a.jacobi ? fma(-alpha, d * si, rtr_[i]) : rn;
      const double pn = fma(beta, pi, rtn);
      double sn = 0.0;
      if (a.dim == 3 && z > 0) sn = fma(-1.0, pnew(i - pl), sn);
      if (y > 0) sn = fma(-1.0, pnew(i - a.nx), sn);
      if (x > 0) sn = fma(-1.0, pnew(i - 1), sn);
      sn = fma(a.cdiag, pnew(i), sn);
      if (x < a.nx - 1) sn = fma(-1.0, pnew(i + 1), sn);
      if (y < a.ny - 1) sn = fma(-1.0, pnew(i + a.nx), sn);
      if (a.dim == 3 && z < a.nz - 1) sn = fma(-1.0, pnew(i + pl), sn);
      const double stn = a.jacobi ? d * sn : sn;
      r[qw][i] = rn;
      rt[qw][i] = rtn;
      p[qw][i] = pn;
      s[qw][i] = sn;
      a5[0] += pn * sn;
      a5[1] += rtn * sn;
      a5[2] += stn * sn;
      a5[3] += rtn * rn;
      a5[4] += rn * rn;
    }
    prcg::block_sum<5>(a5, sm);
    if (tid == 0) {
      mu = a5[0];
      sigma = a5[1];
      gamma = a5[2];
      nu = a5[3];
      const double rel = sqrt(a.jacobi ? a5[4] : a5[3]) / sqrt(st_bn2);
      if (a.hist) a.hist[k] = rel;
      hdr[1] = k;
      if (rel <= a.tol) {
        hdr[0] = 0;
        sc[2] = 0.0;
      } else if (k >= a.maxit) {
        hdr[0] = 1;
        sc[2] = 0.0;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  // b == 0: the solution is x = 0
  if (hdr[2] != 0.0)
    for (int i = tid; i < n; i += kNoallocThreads) a.x[i] = 0.0;
}

// Device address of the scratch array for the current device (set-up on the
// first call per device).
int scratch_for_device(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return PRCG_ERR_CUDA;
  double* ptr = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!ptr) {
    if (cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return PRCG_ERR_CUDA;
    }
    g_scratch_ptr[dev].store(ptr, std::memory_order_release);
  }
  *out = ptr;
  return PRCG_OK;
}

// True for memory the kernel on device `dev` may dereference: device memory
// of `dev` itself, or managed memory.  Device memory of another GPU is
// refused (without peer access a load from it would fault).
bool is_device_pointer(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int prcg_pr_solve_stencil_noalloc(int dim, int64_t nx, int64_t ny, int64_t nz,
                                             double diag_shift, int precond, const double* b,
                                             double* x, double tol, int maxit,
                                             double* residual_history, int* iters_out,
                                             void* cuda_stream) {
  if (dim != 2 && dim != 3) return PRCG_ERR_INVALID;
  if (dim == 2) nz = 1;
  if (nx < 1 || ny < 1 || nz < 1) return PRCG_ERR_INVALID;
  // each extent is bounded before the product is formed, so it cannot overflow
  if (nx > kNoallocMaxN || ny > kNoallocMaxN || nz > kNoallocMaxN) return PRCG_ERR_INVALID;
  if (nx * ny > kNoallocMaxN) return PRCG_ERR_INVALID;
  const int64_t n = nx * ny * nz;
  if (n > kNoallocMaxN) return PRCG_ERR_INVALID;   // beyond the fixed scratch size
  if (precond != PRCG_PRECOND_NONE && precond != PRCG_PRECOND_JACOBI) return PRCG_ERR_INVALID;
  if (!(diag_shift >= 0.0) || !std::isfinite(diag_shift)) return PRCG_ERR_INVALID;
  if (!(tol >= 0.0) || maxit < 0 || !b || !x) return PRCG_ERR_INVALID;
  if ((int64_t)maxit > kNoallocMaxItPerRow * n + kNoallocMaxItExtra) return PRCG_ERR_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PRCG_ERR_CUDA;
  }
  if (!is_device_pointer(b, dev) || !is_device_pointer(x, dev)) return PRCG_ERR_INVALID;
  if (residual_history && !is_device_pointer(residual_history, dev)) return PRCG_ERR_INVALID;
  double* scratch = nullptr;
  if (scratch_for_device(dev, &scratch) != PRCG_OK) return PRCG_ERR_CUDA;
  NoallocArgs a;
  a.dim = dim;
  a.nx = (int)nx;
  a.ny = (int)ny;
  a.nz = (int)nz;
  a.n = (int)n;
  a.cdiag = 2.0 * dim + diag_shift;
  a.jacobi = precond == PRCG_PRECOND_JACOBI;
  a.d = a.jacobi ? 1.0 / a.cdiag : 1.0;
  a.b = b;
  a.x = x;
  a.hist = residual_history;
  a.tol = tol;
  a.maxit = maxit;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_pr_noalloc<<<1, kNoallocThreads, 0, st>>>(a, scratch);
  if (cudaGetLastError() != cudaSuccess) return PRCG_ERR_CUDA;
  double hdr[3] = {0.0, 0.0, 0.0};
  if (cudaMemcpyAsync(hdr, scratch, sizeof hdr, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PRCG_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PRCG_ERR_CUDA;
  const int status = (int)hdr[0];
  if (iters_out) *iters_out = (int)hdr[1];
  if (status == -100) return PRCG_ERR_CUDA;
  return status;
}
