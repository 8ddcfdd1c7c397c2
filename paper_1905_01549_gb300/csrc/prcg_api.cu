// C ABI of the predict-and-recompute CG library (declared in include/prcg.h).
//
// A context owns device copies of the operator, the Jacobi diagonal, the
// iteration vectors (double-buffered where a sweep gathers them), the
// device-resident scalar block and, per variant, one instantiated CUDA
// graph: the initialisation sweeps followed by a device-side while loop
// whose body runs a fixed number of fused iteration sweeps and a one-thread
// kernel that decides whether to go on.  A solve is therefore one graph
// launch with no host round trip per iteration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "../../include/prcg.h"
#include "prcg_launch.cuh"

namespace prcg {
LaunchFn launcher_csr(int op_kind, int pc_kind);
LaunchFn launcher_csr_scalar(int op_kind, int pc_kind);
LaunchFn launcher_st(int op_kind, int pc_kind);
LaunchFn launcher_vc(int op_kind, int pc_kind);
LaunchFn launcher_dense(int op_kind, int pc_kind);

LaunchFn launcher_for(int op_kind, int pc_kind) {
  if ((op_kind == OP_CSR || op_kind == OP_SELL) && pc_kind == PC_SCALAR)
    return launcher_csr_scalar(op_kind, pc_kind);
  if (op_kind == OP_CSR || op_kind == OP_SELL) return launcher_csr(op_kind, pc_kind);
  if (op_kind == OP_ST2 || op_kind == OP_ST3) return launcher_st(op_kind, pc_kind);
  if (op_kind == OP_DENSE) return launcher_dense(op_kind, pc_kind);
  return launcher_vc(op_kind, pc_kind);
}

// ---------------------------------------------------------------- set-up kernels
__global__ void k_check_csr(const int* rp, const int* ci, int n, int nnz, int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e0 = rp[i], e1 = rp[i + 1];
    if (e0 < 0 || e1 < e0 || e1 > nnz) {
      atomicOr(bad, 1);
      continue;
    }
    for (int e = e0; e < e1; ++e) {
      const int j = ci[e];
      if (j < 0 || j >= n) atomicOr(bad, 2);
    }
  }
}

// d_i = 1 / a_ii (Section 4: Jacobi); flags a missing or non-positive a_ii.
__global__ void k_csr_jacobi(const int* rp, const int* ci, const double* va, int n, double* d,
                             int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] == i) a += va[e];
    if (!(a > 0.0) || !isfinite(a)) {
      atomicOr(bad, 4);
      d[i] = 0.0;
    } else {
      d[i] = 1.0 / a;
    }
  }
}

// Flags (bit 8) a Jacobi diagonal that is not one constant: d_i != d_0
// bitwise for some i.
__global__ void k_const_diag(const double* d, int n, int* flag) {
  const unsigned long long d0 = __double_as_longlong(d[0]);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if ((unsigned long long)__double_as_longlong(d[i]) != d0) {
      atomicOr(flag, 8);
      return;
    }
}

// Guard bands: 256-byte blocks after every vector and partial-sum buffer,
// filled with a signalling-NaN bit pattern (FP64 arithmetic only ever
// produces quiet NaNs, so no computed value matches it).  An out-of-bounds
// write by any kernel changes a guard word; prcg_check_guards counts them.
constexpr int kGuardWords = 32;
constexpr unsigned long long kGuardPattern = 0x7FF4DEADBEEFCAFEull;

__global__ void k_guard_fill(unsigned long long* p, size_t cnt) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt;
       i += (size_t)gridDim.x * blockDim.x)
    p[i] = kGuardPattern;
}

__global__ void k_guard_count(const unsigned long long* p, size_t cnt, unsigned long long* bad) {
  unsigned long long m = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt;
       i += (size_t)gridDim.x * blockDim.x)
    m += p[i] != kGuardPattern;
  if (m) atomicAdd(bad, m);
}

// d_i = 1 / a_ii of a dense matrix (column-major, leading dimension lda).
__global__ void k_dense_jacobi(const double* A, int n, int lda, double* d, int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = A[(size_t)i * lda + i];
    if (!(a > 0.0) || !isfinite(a))
      atomicOr(bad, 4);
    else
      d[i] = 1.0 / a;
  }
}

// SELL-32 conversion: entries per row of each 32-row slice (the slice max).
__global__ void k_sell_len(const int* rp, int n, int nslices, int* slen) {
  for (int sl = blockIdx.x * blockDim.x + threadIdx.x; sl < nslices; sl += gridDim.x * blockDim.x) {
    int L = 0;
    for (int l = 0; l < 32; ++l) {
      const int i = sl * 32 + l;
      if (i < n) L = max(L, rp[i + 1] - rp[i]);
    }
    slen[sl] = L;
  }
}

// SELL-32 fill: entry t of row i goes to sptr[i/32] + 32 t + i%32; padding
// entries (and the rows past n in the last slice) point at a valid column
// with value 0.
__global__ void k_sell_fill(const int* rp, const int* ci, const double* va, int n, int nslices,
                            const int* sptr, const int* slen, int* scol, double* sval) {
  const int total = nslices * 32;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int sl = i >> 5, l = i & 31;
    const int L = slen[sl];
    const int base = sptr[sl] + l;
    const int e0 = i < n ? rp[i] : 0;
    const int len = i < n ? rp[i + 1] - e0 : 0;
    const int pad_col = i < n ? i : n - 1;
    for (int t = 0; t < L; ++t) {
      const int e = base + 32 * t;
      if (t < len) {
        scol[e] = ci[e0 + t];
        sval[e] = va[e0 + t];
      } else {
        scol[e] = pad_col;
        sval[e] = 0.0;
      }
    }
  }
}

// Diagonal of the variable-coefficient operator: the sum of the cell's face
// coefficients (x-, x+, y-, y+, z-, z+) plus the shift; optionally 1 / a_ii.
__global__ void k_vc_diag(int dim, int nx, int ny, int nz, const double* fx, const double* fy,
                          const double* fz, double shift, double* adiag, double* d, int* bad) {
  const int n = nx * ny * nz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int x = i % nx, yz = i / nx, y = yz % ny, z = yz / ny;
    double a = fx[yz * (nx + 1) + x] + fx[yz * (nx + 1) + x + 1];
    a = a + fy[(z * (ny + 1) + y) * nx + x];
    a = a + fy[(z * (ny + 1) + y + 1) * nx + x];
    if (dim == 3) {
      a = a + fz[i];
      a = a + fz[i + nx * ny];
    }
    a = a + shift;
    adiag[i] = a;
    if (d) {
      if (!(a > 0.0) || !isfinite(a)) {
        atomicOr(bad, 4);
        d[i] = 0.0;
      } else {
        d[i] = 1.0 / a;
      }
    }
  }
}

// v_i = 0.5 + u_i with u_i in [0, 1) from the SplitMix64 finaliser of i
// (Steele, Lea and Flood, OOPSLA 2014): a fixed right-hand side with no
// structure, so that every row of every iterate is nonzero from the first
// iteration on.
__global__ void k_fill_hashed(double* v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = 0.5 + (double)(z >> 11) * 0x1p-53;
  }
}

// Adjoint gradient of the face coefficients: for x = A^{-1} b and lambda =
// A^{-1} dL/dx, dL/dc_f = -(lambda_a - lambda_b)(x_a - x_b) for the interior
// face between cells a and b, and -lambda_a x_a for a boundary face of cell a.
__global__ void k_grad_faces(int dim, int nx, int ny, int nz, const double* lam, const double* x,
                             double* g) {
  const long long nfx = (long long)nz * ny * (nx + 1);
  const long long nfy = (long long)nz * (ny + 1) * nx;
  const long long nfz = dim == 3 ? (long long)(nz + 1) * ny * nx : 0;
  const long long nf = nfx + nfy + nfz;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf;
       f += (long long)gridDim.x * blockDim.x) {
    long long a = -1, b = -1;
    if (f < nfx) {
      const long long fx = f % (nx + 1), yz = f / (nx + 1);
      const long long base = yz * nx;
      if (fx > 0) a = base + fx - 1;
      if (fx < nx) b = base + fx;
    } else if (f < nfx + nfy) {
      const long long q = f - nfx;
      const long long x0 = q % nx, t = q / nx, fy = t % (ny + 1), z = t / (ny + 1);
      if (fy > 0) a = (z * ny + fy - 1) * nx + x0;
      if (fy < ny) b = (z * ny + fy) * nx + x0;
    } else {
      const long long q = f - nfx - nfy;
      const long long pl = (long long)nx * ny;
      const long long fz = q / pl, xy = q % pl;
      if (fz > 0) a = (fz - 1) * pl + xy;
      if (fz < nz) b = fz * pl + xy;
    }
    double v;
    if (a >= 0 && b >= 0)
      v = -(lam[a] - lam[b]) * (x[a] - x[b]);
    else {
      const long long c = a >= 0 ? a : b;
      v = -lam[c] * x[c];
    }
    g[f] = v;
  }
}

// dL/da_ij = -lambda_i x_j for every stored entry (caller's CSR order).
__global__ void k_grad_csr(const int* rp, const int* ci, int n, const double* lam, const double* x,
                           double* g) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double li = lam[i];
    for (int e = rp[i]; e < rp[i + 1]; ++e) g[e] = -li * x[ci[e]];
  }
}

__global__ void k_to_f32(const double* a, float* b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Body-end control of the device-side while loop.
__global__ void k_loop_control(cudaGraphConditionalHandle h, DevState* S) {
  const unsigned b = S->bodies + 1u;
  S->bodies = b;
  bool more = S->done == 0;
  if (more && (int)b >= S->maxbodies) {
    S->status = PRCG_ERR_TIMEOUT;
    S->done = 1;
    more = false;
  }
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

}  // namespace prcg

using namespace prcg;

namespace {

thread_local std::string g_create_error;

struct VariantGraph {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int chunk = 0;
};

}  // namespace

struct prcg_ctx {
  int device = 0;
  cudaStream_t user = nullptr;
  cudaStream_t cs = nullptr;     // internal stream all work runs on
  cudaStream_t bs = nullptr;     // capture stream for loop bodies
  cudaEvent_t ev_user = nullptr, ev_start = nullptr, ev_init = nullptr, ev_loop = nullptr;
  Plan plan{};
  LaunchFn launch = nullptr;
  int n = 0;
  int precond = 0;
  double* pool = nullptr;        // all n-length vectors
  int* ipool = nullptr;          // CSR indices
  double* vpool = nullptr;       // CSR values / faces / diagonals
  int* sell_i = nullptr;         // SELL-32 slice pointers, lengths, columns
  double* sell_v = nullptr;      // SELL-32 values
  double* partials = nullptr;
  DevState* S = nullptr;
  DevState* hS = nullptr;        // pinned mirror
  double* hist = nullptr;
  int hist_cap = 0;
  int* dbad = nullptr;
  VariantGraph graphs[10];
  bool use_graph = true;
  float t_init = 0.f, t_loop = 0.f;
  int last_iters = 0;
  int64_t last_launches = 0;
  int64_t last_pf_sweeps = 0;   // product sweeps of the last solve that read the fixed-point p
  int64_t host_loop_launches = 0;
  float* pool32 = nullptr;       // FP32 vectors of the mixed-precision inner solve
  float* sval32 = nullptr;       // FP32 copy of the SELL values
  DevState* S2 = nullptr;        // scalar block of the inner solve
  GridBar* gb = nullptr;         // grid barrier of the persistent solve
  int persist_max = 1 << 21;     // largest n solved by the persistent kernel
  bool trace_on = false;         // record the scalar trace of each solve
  double* trace = nullptr;       // device, trace_cap slots x kTraceFields
  int trace_cap = 0;
  int trace_slots = 0;           // slots written by the last solve (K + 1)
  std::vector<std::pair<void*, size_t>> guards;   // guard bands (pointer, 8-byte words)
  GridBar hgb{};                 // host image of the barrier state of the next persistent launch
  bool inject_once = false;      // hgb carries a one-shot failure injection
  unsigned long long* dguard = nullptr;           // device counter of corrupted guard words
  double* gscratch = nullptr;    // face-gradient scratch (variable-coefficient stencils)
  std::string err;
};

namespace {

int set_err(prcg_ctx* c, int code, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_error = msg;
  return code;
}

int cuda_err(prcg_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return set_err(c, e == cudaErrorMemoryAllocation ? PRCG_ERR_OOM : PRCG_ERR_CUDA, m);
}

#define CK(call)                                    \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_err(c, e_, #call); \
  } while (0)

// The constant-stencil product sweeps of HS-CG and PR-CG read a block
// fixed-point copy of p unless PRCG_NO_FIXED_P=1 (then the per-row
// fixed-point neighbour sums are used).
int fixed_p_allowed() {
  const char* e = getenv("PRCG_NO_FIXED_P");
  return (e && e[0] == '1') ? 0 : 1;
}

// Register and fill a guard band of `words` 8-byte words at p.
int add_guard(prcg_ctx* c, void* p, size_t words) {
  c->guards.emplace_back(p, words);
  k_guard_fill<<<1, 256, 0, c->cs>>>(static_cast<unsigned long long*>(p), words);
  CK(cudaGetLastError());
  return PRCG_OK;
}

int ctx_init_common(prcg_ctx* c, void* stream, int n) {
  c->n = n;
  c->user = (cudaStream_t)stream;
  CK(cudaGetDevice(&c->device));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  c->plan.sms = sms;
  CK(cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&c->bs, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming));
  CK(cudaEventCreate(&c->ev_start));
  CK(cudaEventCreate(&c->ev_init));
  CK(cudaEventCreate(&c->ev_loop));
  // 23 n-vectors: x, b, t, d, two buffers each of r, r~, p, s, s~, w, u, and
  // the block fixed-point copies (64-bit integers) of p and, per buffer, of
  // r~ and s~; each starts on a 256-byte boundary and is followed by a guard
  // band that covers its rounding up to 32 entries and 32 more words
  const size_t nv = 23;
  const size_t nr = ((size_t)n + 31) / 32 * 32, stride = nr + kGuardWords;
  CK(cudaMalloc(&c->pool, (kGuardWords + nv * stride) * sizeof(double)));
  int grc = add_guard(c, c->pool, kGuardWords);
  double* q = c->pool + kGuardWords;
  size_t taken = 0;
  auto take = [&]() {
    double* r = q;
    if (grc == PRCG_OK) grc = add_guard(c, r + n, stride - (size_t)n);
    q += stride;
    ++taken;
    return r;
  };
  Vecs& V = c->plan.v;
  V.x = take();
  V.b = take();
  V.t = take();
  V.pf = reinterpret_cast<long long*>(take());
  for (int bq = 0; bq < 2; ++bq) {
    V.rtf[bq] = reinterpret_cast<long long*>(take());
    V.stf[bq] = reinterpret_cast<long long*>(take());
  }
  double* d = take();
  for (int k = 0; k < 2; ++k) {
    V.r[k] = take();
    V.rt[k] = take();
    V.p[k] = take();
    V.s[k] = take();
    V.st[k] = take();
    V.w[k] = take();
    V.u[k] = take();
  }
  c->plan.pc.d = d;
  if (taken != nv) return set_err(c, PRCG_ERR_INVALID, "internal: vector pool size mismatch");
  if (grc != PRCG_OK) return grc;
  // partial sums: kMaxGrid x (kMaxNV + 2) for the sweeps, and two epochs of
  // kMaxPersistCtas x 8 for the persistent solve's barriers (the larger)
  const size_t npart = std::max((size_t)kMaxGrid * (kMaxNV + 2), (size_t)2 * kMaxPersistCtas * 8);
  CK(cudaMalloc(&c->partials, (npart + kGuardWords) * sizeof(double)));
  if ((grc = add_guard(c, c->partials + npart, kGuardWords)) != PRCG_OK) return grc;
  CK(cudaMalloc(&c->dguard, sizeof(unsigned long long)));
  CK(cudaMalloc(&c->S, sizeof(DevState)));
  CK(cudaMemset(c->S, 0, sizeof(DevState)));
  CK(cudaMallocHost(&c->hS, sizeof(DevState)));
  CK(cudaMalloc(&c->dbad, sizeof(int)));
  CK(cudaMemset(c->dbad, 0, sizeof(int)));
  c->plan.S = c->S;
  c->plan.partials = c->partials;
  c->plan.partials_a = c->partials + (size_t)kMaxGrid * kMaxNV;
  CK(cudaMalloc(&c->gb, sizeof(GridBar)));
  c->plan.gb = c->gb;
  const char* ng = getenv("PRCG_NO_GRAPH");
  c->use_graph = !(ng && ng[0] == '1');
  const char* pm = getenv("PRCG_PERSIST_MAX");
  if (pm) c->persist_max = atoi(pm);
  return PRCG_OK;
}

// Order the internal stream after everything already queued on the user's.
int wait_user(prcg_ctx* c) {
  CK(cudaEventRecord(c->ev_user, c->user));
  CK(cudaStreamWaitEvent(c->cs, c->ev_user, 0));
  return PRCG_OK;
}

int check_bad(prcg_ctx* c, const char* what) {
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, c->dbad, sizeof(int), cudaMemcpyDeviceToHost, c->cs));
  CK(cudaStreamSynchronize(c->cs));
  if (bad) {
    char m[160];
    snprintf(m, sizeof m, "%s (flags %d: 1 row_ptr, 2 col_idx, 4 diagonal)", what, bad);
    return set_err(c, PRCG_ERR_INVALID, m);
  }
  return PRCG_OK;
}

void destroy_graphs(prcg_ctx* c) {
  for (auto& g : c->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g.exec = nullptr;
    g.graph = nullptr;
  }
}

int launch_init(prcg_ctx* c, int variant, cudaStream_t st) {
  CK(c->launch(c->plan, PH_INIT_A, variant, 0, 0, st));
  CK(c->launch(c->plan, PH_INIT_B, variant, 0, 0, st));
  return PRCG_OK;
}

int init_launches(int) { return 2; }

// Extra kernels per product sweep: dense operators form each product in a
// pre-pass launch.
int product_prepasses(const prcg_ctx* c) { return c->plan.op.kind == OP_DENSE ? 1 : 0; }

// Kernels of one iteration of `variant`.
int iter_launches(int variant) {
  switch (variant) {
    case V_HS: return 3;
    case V_PR:
    case V_M:
    case V_PR_NR:
    case V_CGCG: return 2;
    default: return 1;
  }
}

// One iteration of `variant`; the pipelined sweep reads buffer qr and
// writes buffer qw.
int launch_iter(prcg_ctx* c, int variant, int qr, int qw, cudaStream_t st) {
  switch (variant) {
    case V_HS:
      CK(c->launch(c->plan, PH_HS_A, variant, qr, qw, st));
      CK(c->launch(c->plan, PH_HS_B, variant, qr, qw, st));
      CK(c->launch(c->plan, PH_HS_C, variant, qr, qw, st));
      break;
    case V_PR:
    case V_M:
    case V_PR_NR:
      CK(c->launch(c->plan, PH_PR_A, variant, qr, qw, st));
      CK(c->launch(c->plan, PH_PR_B, variant, qr, qw, st));
      break;
    case V_PIPE:
    case V_PIPE_M:
      CK(c->launch(c->plan, PH_PIPE, variant, qr, qw, st));
      break;
    case V_CGCG:
      CK(c->launch(c->plan, PH_CG_A, variant, qr, qw, st));
      CK(c->launch(c->plan, PH_CG_B, variant, qr, qw, st));
      break;
    case V_GV:
      CK(c->launch(c->plan, PH_GV, variant, qr, qw, st));
      break;
    case V_PIPE_NR:
      CK(c->launch(c->plan, PH_PIPE_NR, variant, qr, qw, st));
      break;
    default:
      return set_err(c, PRCG_ERR_UNSUPPORTED, "variant not built on the GPU path");
  }
  return PRCG_OK;
}

int chunk_for(prcg_ctx* c) { return c->n >= (1 << 20) ? 2 : 16; }

constexpr int kMixedGraph = 9;   // graphs[9]: the FP32 inner solve of the mixed form

int launch_mixed_init(prcg_ctx* c, cudaStream_t st) {
  CK(c->launch(c->plan, PH_MX_INIT_A, 0, 0, 0, st));
  CK(c->launch(c->plan, PH_MX_INIT_B, 0, 0, 0, st));
  return PRCG_OK;
}

int launch_mixed_iter(prcg_ctx* c, cudaStream_t st) {
  CK(c->launch(c->plan, PH_MX_PR_A, 0, 0, 0, st));
  CK(c->launch(c->plan, PH_MX_PR_B, 0, 0, 0, st));
  return PRCG_OK;
}

int build_graph(prcg_ctx* c, int variant) {
  VariantGraph& G = c->graphs[variant];
  if (G.exec) return PRCG_OK;
  const bool mixed = variant == kMixedGraph;
  DevState* SS = mixed ? c->S2 : c->S;
  const int chunk = chunk_for(c);
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  G.graph = g;
  CK(cudaStreamBeginCaptureToGraph(c->cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  int rc = mixed ? launch_mixed_init(c, c->cs) : launch_init(c, variant, c->cs);
  if (rc == PRCG_OK) {
    cudaError_t e = cudaEventRecordWithFlags(c->ev_init, c->cs, cudaEventRecordExternal);
    if (e != cudaSuccess) rc = cuda_err(c, e, "event record in capture");
  }
  cudaGraphConditionalHandle h;
  cudaGraphNode_t cond = nullptr;
  if (rc == PRCG_OK) {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaGraph_t cg = nullptr;
    cudaError_t e = cudaStreamGetCaptureInfo(c->cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cond, g, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess)
      e = cudaStreamUpdateCaptureDependencies(c->cs, &cond, nullptr, 1,
                                              cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) {
      rc = cuda_err(c, e, "conditional node");
    } else {
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      e = cudaStreamBeginCaptureToGraph(c->bs, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) rc = cuda_err(c, e, "body capture");
      for (int m = 0; rc == PRCG_OK && m < chunk; ++m)
        rc = mixed ? launch_mixed_iter(c, c->bs) : launch_iter(c, variant, m & 1, (m + 1) & 1, c->bs);
      if (rc == PRCG_OK) {
        k_loop_control<<<1, 1, 0, c->bs>>>(h, SS);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_err(c, e, "loop control launch");
      }
      cudaGraph_t bo = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(c->bs, &bo);
      if (rc == PRCG_OK && e2 != cudaSuccess) rc = cuda_err(c, e2, "end body capture");
    }
  }
  if (rc == PRCG_OK) {
    cudaError_t e = cudaEventRecordWithFlags(c->ev_loop, c->cs, cudaEventRecordExternal);
    if (e != cudaSuccess) rc = cuda_err(c, e, "event record in capture");
  }
  cudaGraph_t go = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(c->cs, &go);
  if (rc == PRCG_OK && e3 != cudaSuccess) rc = cuda_err(c, e3, "end capture");
  if (rc == PRCG_OK) {
    cudaError_t e = cudaGraphInstantiate(&G.exec, g, 0);
    if (e != cudaSuccess) rc = cuda_err(c, e, "graph instantiate");
  }
  if (rc != PRCG_OK) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    cudaGraphDestroy(g);
    G.exec = nullptr;
    G.graph = nullptr;
    cudaGetLastError();
    return rc;
  }
  G.chunk = chunk;
  return PRCG_OK;
}

// Host-driven loop, used when graphs are disabled (PRCG_NO_GRAPH=1) or fail
// to build: the same sweeps launched directly, with the status read back
// after every chunk.
int run_host_loop(prcg_ctx* c, int variant, int maxit) {
  const int chunk = chunk_for(c);
  int rc = launch_init(c, variant, c->cs);
  if (rc != PRCG_OK) return rc;
  CK(cudaEventRecord(c->ev_init, c->cs));
  for (int it = 0; it <= maxit; it += chunk) {
    CK(cudaMemcpyAsync(c->hS, c->S, sizeof(DevState), cudaMemcpyDeviceToHost, c->cs));
    CK(cudaStreamSynchronize(c->cs));
    if (c->hS->done) break;
    for (int m = 0; m < chunk; ++m) {
      rc = launch_iter(c, variant, m & 1, (m + 1) & 1, c->cs);
      if (rc != PRCG_OK) return rc;
      c->host_loop_launches += iter_launches(variant) + product_prepasses(c);
    }
  }
  CK(cudaEventRecord(c->ev_loop, c->cs));
  return PRCG_OK;
}

// Re-lay the validated CSR matrix out as SELL-32 (padding at most doubles
// the stored entries; otherwise the CSR layout is kept).
int build_sell(prcg_ctx* c) {
  OpDesc& op = c->plan.op;
  const int n = op.n;
  const int nslices = (n + 31) / 32;
  int* slen_d = nullptr;
  CK(cudaMalloc(&slen_d, (size_t)nslices * sizeof(int)));
  k_sell_len<<<c->plan.sms * 4, 256, 0, c->cs>>>(op.rp, n, nslices, slen_d);
  std::vector<int> slen(nslices);
  cudaError_t e = cudaMemcpyAsync(slen.data(), slen_d, (size_t)nslices * sizeof(int),
                                  cudaMemcpyDeviceToHost, c->cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->cs);
  cudaFree(slen_d);
  if (e != cudaSuccess) return cuda_err(c, e, "SELL lengths");
  std::vector<int> sptr(nslices + 1);
  int64_t total = 0;
  for (int sl = 0; sl < nslices; ++sl) {
    sptr[sl] = (int)total;
    total += 32 * (int64_t)slen[sl];
    if (total >= ((int64_t)1 << 31) - 64) return PRCG_OK;  // keep CSR
  }
  sptr[nslices] = (int)total;
  int nnz = 0;
  CK(cudaMemcpy(&nnz, op.rp + n, sizeof(int), cudaMemcpyDeviceToHost));
  if (total > 2 * (int64_t)nnz + 64 * (int64_t)nslices) return PRCG_OK;  // too much padding
  // columns start on a 128-byte boundary: TMA copies whole tiles of them
  const size_t col_off = ((size_t)(2 * nslices + 1) + 31) / 32 * 32;
  const size_t ni = col_off + (size_t)total + 4;
  CK(cudaMalloc(&c->sell_i, ni * sizeof(int)));
  CK(cudaMalloc(&c->sell_v, ((size_t)total + 2) * sizeof(double)));
  int* sptr_d = c->sell_i;
  int* slen2_d = c->sell_i + nslices + 1;
  int* scol_d = c->sell_i + col_off;
  CK(cudaMemcpyAsync(sptr_d, sptr.data(), (size_t)(nslices + 1) * sizeof(int),
                     cudaMemcpyHostToDevice, c->cs));
  CK(cudaMemcpyAsync(slen2_d, slen.data(), (size_t)nslices * sizeof(int), cudaMemcpyHostToDevice,
                     c->cs));
  k_sell_fill<<<c->plan.sms * 8, 256, 0, c->cs>>>(op.rp, op.ci, op.va, n, nslices, sptr_d, slen2_d,
                                                 scol_d, c->sell_v);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->cs));
  op.sptr = sptr_d;
  op.slen = slen2_d;
  op.scol = scol_d;
  op.sval = c->sell_v;
  op.kind = OP_SELL;
  const char* nt = getenv("PRCG_NO_TMA");
  op.tma = (!(nt && nt[0] == '1') && sell_fits_tma(sptr.data(), nslices)) ? 1 : 0;
  return PRCG_OK;
}

int copy_in(prcg_ctx* c, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->cs));
  return PRCG_OK;
}

// The caller's concatenated face array (x-faces, y-faces, z-faces) into the
// context's three aligned face arrays.
int copy_faces(prcg_ctx* c, const OpDesc& op, const double* faces, size_t nfx, size_t nfy,
               size_t nfz) {
  int rc;
  if ((rc = copy_in(c, const_cast<double*>(op.fx), faces, nfx * sizeof(double))) != PRCG_OK)
    return rc;
  if ((rc = copy_in(c, const_cast<double*>(op.fy), faces + nfx, nfy * sizeof(double))) != PRCG_OK)
    return rc;
  if (nfz)
    rc = copy_in(c, const_cast<double*>(op.fz), faces + nfx + nfy, nfz * sizeof(double));
  return rc;
}

// Test kernel: the stencil operators' neighbour sum over count K-tuples.
template <int K>
__global__ void k_test_neighbour_sum(const double* __restrict__ v, int64_t count,
                                     double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    double a[K];
#pragma unroll
    for (int j = 0; j < K; ++j) a[j] = v[t * K + j];
    out[t] = neighbour_sum<K>(a);
  }
}

// Host spot check of the invariant-divisor quotient the stencil sweeps use
// for every dividend 0 <= v < limit: the end points, and the neighbourhood of
// the multiples of d near the top of the range, where a wrong multiplier
// fails first.
bool fastdiv_ok(const FastDiv& f, int d, int limit) {
  auto ok = [&](long long v) {
    return v < 0 || v >= limit || fast_div(f, (int)v) == (int)(v / d);
  };
  if (!ok(0) || !ok(limit - 1)) return false;
  const long long top = (long long)(limit - 1) / d;
  for (long long q = top; q >= 0 && q > top - 64; --q)
    for (long long e = -2; e <= 2; ++e)
      if (!ok(q * d + e)) return false;
  for (long long q = 0; q < 64; ++q)
    for (long long e = -2; e <= 2; ++e)
      if (!ok(q * d + e)) return false;
  return true;
}

}  // namespace

extern "C" {

int prcg_create_csr(prcg_ctx** out, int64_t n, int64_t nnz, const int32_t* row_ptr,
                    const int32_t* col_idx, const double* vals, int precond, void* cuda_stream) {
  prcg_ctx* c = nullptr;
  if (!out) return set_err(nullptr, PRCG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1 || n >= (int64_t)1 << 31 || nnz < 0 || nnz >= (int64_t)1 << 31)
    return set_err(nullptr, PRCG_ERR_INVALID, "n or nnz out of range");
  if (!row_ptr || (nnz > 0 && (!col_idx || !vals)))
    return set_err(nullptr, PRCG_ERR_INVALID, "NULL array");
  if (precond != PRCG_PRECOND_NONE && precond != PRCG_PRECOND_JACOBI)
    return set_err(nullptr, PRCG_ERR_INVALID, "unknown preconditioner");
  c = new prcg_ctx();
  int rc = ctx_init_common(c, cuda_stream, (int)n);
  if (rc != PRCG_OK) {
    g_create_error = c->err;
    prcg_destroy(c);
    return rc;
  }
  auto fail = [&](int code) {
    g_create_error = c->err;
    prcg_destroy(c);
    return code;
  };
  const size_t idx_elems = (size_t)(n + 1) + (size_t)nnz + 4;  // +4: room for vector loads
  if (cudaMalloc(&c->ipool, idx_elems * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&c->vpool, ((size_t)nnz + 2) * sizeof(double)) != cudaSuccess)
    return fail(set_err(c, PRCG_ERR_OOM, "CSR allocation failed"));
  int* rp = c->ipool;
  int* ci = c->ipool + (n + 1);
  double* va = c->vpool;
  if ((rc = wait_user(c)) != PRCG_OK) return fail(rc);
  if ((rc = copy_in(c, rp, row_ptr, (size_t)(n + 1) * sizeof(int))) != PRCG_OK) return fail(rc);
  if (nnz > 0) {
    if ((rc = copy_in(c, ci, col_idx, (size_t)nnz * sizeof(int))) != PRCG_OK) return fail(rc);
    if ((rc = copy_in(c, va, vals, (size_t)nnz * sizeof(double))) != PRCG_OK) return fail(rc);
  }
  int ends[2] = {0, 0};
  cudaMemcpyAsync(&ends[0], rp, sizeof(int), cudaMemcpyDeviceToHost, c->cs);
  cudaMemcpyAsync(&ends[1], rp + n, sizeof(int), cudaMemcpyDeviceToHost, c->cs);
  if (cudaStreamSynchronize(c->cs) != cudaSuccess) return fail(cuda_err(c, cudaGetLastError(), "copy"));
  if (ends[0] != 0 || ends[1] != nnz) return fail(set_err(c, PRCG_ERR_INVALID, "row_ptr[0] != 0 or row_ptr[n] != nnz"));
  k_check_csr<<<c->plan.sms * 4, 256, 0, c->cs>>>(rp, ci, (int)n, (int)nnz, c->dbad);
  if ((rc = check_bad(c, "invalid CSR structure")) != PRCG_OK) return fail(rc);
  c->plan.op.kind = OP_CSR;
  c->plan.op.n = (int)n;
  c->plan.op.rp = rp;
  c->plan.op.ci = ci;
  c->plan.op.va = va;
  c->precond = precond;
  c->plan.pc.kind = PC_NONE;
  if (precond == PRCG_PRECOND_JACOBI) {
    c->plan.pc.kind = PC_VEC;
    k_csr_jacobi<<<c->plan.sms * 4, 256, 0, c->cs>>>(rp, ci, va, (int)n,
                                                    const_cast<double*>(c->plan.pc.d), c->dbad);
    if ((rc = check_bad(c, "Jacobi needs a positive diagonal")) != PRCG_OK) return fail(rc);
    // A diagonal that is one constant (every d_i bitwise equal) is applied as
    // a scalar: the product d_i v_i is the same, the sweeps stop reading d,
    // and d folds into alpha where a recurrence subtracts alpha M^{-1} v.
    const char* nsc = getenv("PRCG_NO_SCALAR_D");
    if (!(nsc && nsc[0] == '1')) {
      int flag = 0;
      double d0 = 0.0;
      if (cudaMemsetAsync(c->dbad, 0, sizeof(int), c->cs) != cudaSuccess)
        return fail(cuda_err(c, cudaGetLastError(), "memset"));
      k_const_diag<<<c->plan.sms * 4, 256, 0, c->cs>>>(c->plan.pc.d, (int)n, c->dbad);
      cudaMemcpyAsync(&flag, c->dbad, sizeof(int), cudaMemcpyDeviceToHost, c->cs);
      cudaMemcpyAsync(&d0, c->plan.pc.d, sizeof(double), cudaMemcpyDeviceToHost, c->cs);
      if (cudaStreamSynchronize(c->cs) != cudaSuccess)
        return fail(cuda_err(c, cudaGetLastError(), "constant-diagonal check"));
      if (cudaMemsetAsync(c->dbad, 0, sizeof(int), c->cs) != cudaSuccess)
        return fail(cuda_err(c, cudaGetLastError(), "memset"));
      if (flag == 0) {
        c->plan.pc.kind = PC_SCALAR;
        c->plan.pc.dscalar = d0;
      }
    }
  }
  const char* ns = getenv("PRCG_NO_SELL");
  if (!(ns && ns[0] == '1')) {
    if ((rc = build_sell(c)) != PRCG_OK) return fail(rc);
  }
  c->launch = launcher_for(c->plan.op.kind, c->plan.pc.kind);
  if (!c->launch) return fail(set_err(c, PRCG_ERR_UNSUPPORTED, "operator not built"));
  *out = c;
  return PRCG_OK;
}

int prcg_create_stencil(prcg_ctx** out, int dim, int64_t nx, int64_t ny, int64_t nz,
                        const double* face_coeff, double diag_shift, int precond,
                        void* cuda_stream) {
  if (!out) return set_err(nullptr, PRCG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (dim != 2 && dim != 3) return set_err(nullptr, PRCG_ERR_INVALID, "dim must be 2 or 3");
  if (dim == 2) nz = 1;
  if (nx < 1 || ny < 1 || nz < 1) return set_err(nullptr, PRCG_ERR_INVALID, "grid size < 1");
  const int64_t n = nx * ny * nz;
  if (n + nx * ny >= (int64_t)1 << 31 || nx >= (1 << 30) || ny >= (1 << 30))
    return set_err(nullptr, PRCG_ERR_INVALID, "grid too large");
  if (precond != PRCG_PRECOND_NONE && precond != PRCG_PRECOND_JACOBI)
    return set_err(nullptr, PRCG_ERR_INVALID, "unknown preconditioner");
  if (!(diag_shift >= 0.0) || !std::isfinite(diag_shift))
    return set_err(nullptr, PRCG_ERR_INVALID, "diag_shift must be finite and >= 0");
  prcg_ctx* c = new prcg_ctx();
  int rc = ctx_init_common(c, cuda_stream, (int)n);
  auto fail = [&](int code) {
    g_create_error = c->err;
    prcg_destroy(c);
    return code;
  };
  if (rc != PRCG_OK) return fail(rc);
  OpDesc& op = c->plan.op;
  op.n = (int)n;
  op.nx = (int)nx;
  op.ny = (int)ny;
  op.nz = (int)nz;
  op.divx = make_fastdiv(op.nx);
  op.divy = make_fastdiv(op.ny);
  if (!fastdiv_ok(op.divx, op.nx, op.n) || !fastdiv_ok(op.divy, op.ny, op.n / op.nx))
    return fail(set_err(c, PRCG_ERR_INVALID, "internal: stencil coordinate division check failed"));
  c->precond = precond;
  if (!face_coeff) {
    op.kind = dim == 2 ? OP_ST2 : OP_ST3;
    op.cdiag = 2.0 * dim + diag_shift;
    // a small integer diagonal (Poisson, or an integer shift): the product
    // sweeps that read the block fixed-point copy of p form the whole row in
    // 64-bit integers (|cint P_i| + |sum P_j| < 14 * 2^58)
    // (PRCG_NO_INT_DIAG=1 keeps the FP64 FMA c p_i - sum)
    const char* nid = getenv("PRCG_NO_INT_DIAG");
    const bool int_ok = !(nid && nid[0] == '1');
    op.cint = (int_ok && op.cdiag >= 1.0 && op.cdiag <= 8.0 && op.cdiag == std::floor(op.cdiag))
                  ? (int)op.cdiag
                  : 0;
    c->plan.pc.kind = PC_NONE;
    if (precond == PRCG_PRECOND_JACOBI) {
      c->plan.pc.kind = PC_SCALAR;
      c->plan.pc.dscalar = 1.0 / op.cdiag;
    }
  } else {
    op.kind = dim == 2 ? OP_VC2 : OP_VC3;
    const size_t nfx = (size_t)nz * ny * (nx + 1), nfy = (size_t)nz * (ny + 1) * nx;
    const size_t nfz = dim == 3 ? (size_t)(nz + 1) * ny * nx : 0;
    // each face array and the diagonal start on a 256-byte boundary (the
    // two-row products load y- and z-faces and diagonals as 16-byte pairs)
    auto up32 = [](size_t v) { return (v + 31) / 32 * 32; };
    const size_t ofy = up32(nfx), ofz = ofy + up32(nfy), oad = ofz + up32(nfz);
    if (cudaMalloc(&c->vpool, (oad + up32((size_t)n) + 2) * sizeof(double)) != cudaSuccess)
      return fail(set_err(c, PRCG_ERR_OOM, "face allocation failed"));
    op.fx = c->vpool;
    op.fy = c->vpool + ofy;
    op.fz = dim == 3 ? c->vpool + ofz : nullptr;
    if ((rc = wait_user(c)) != PRCG_OK) return fail(rc);
    if ((rc = copy_faces(c, op, face_coeff, nfx, nfy, nfz)) != PRCG_OK) return fail(rc);
    double* adiag = c->vpool + oad;
    op.adiag = adiag;
    double* d = precond == PRCG_PRECOND_JACOBI ? const_cast<double*>(c->plan.pc.d) : nullptr;
    k_vc_diag<<<c->plan.sms * 4, 256, 0, c->cs>>>(dim, (int)nx, (int)ny, (int)nz, op.fx, op.fy,
                                                 op.fz, diag_shift, adiag, d, c->dbad);
    if ((rc = check_bad(c, "Jacobi needs a positive diagonal")) != PRCG_OK) return fail(rc);
    c->plan.pc.kind = precond == PRCG_PRECOND_JACOBI ? PC_VEC : PC_NONE;
  }
  c->launch = launcher_for(op.kind, c->plan.pc.kind);
  if (!c->launch) return fail(set_err(c, PRCG_ERR_UNSUPPORTED, "operator not built"));
  *out = c;
  return PRCG_OK;
}

int prcg_create_dense(prcg_ctx** out, int64_t n, const double* A, int precond, void* cuda_stream) {
  if (!out) return set_err(nullptr, PRCG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > kMaxDenseN) return set_err(nullptr, PRCG_ERR_INVALID, "n out of range");
  if (!A) return set_err(nullptr, PRCG_ERR_INVALID, "A is NULL");
  if (precond != PRCG_PRECOND_NONE && precond != PRCG_PRECOND_JACOBI)
    return set_err(nullptr, PRCG_ERR_INVALID, "unknown preconditioner");
  prcg_ctx* c = new prcg_ctx();
  int rc = ctx_init_common(c, cuda_stream, (int)n);
  auto fail = [&](int code) {
    g_create_error = c->err;
    prcg_destroy(c);
    return code;
  };
  if (rc != PRCG_OK) return fail(rc);
  OpDesc& op = c->plan.op;
  op.kind = OP_DENSE;
  op.n = (int)n;
  op.lda = (int)((n + 31) / 32 * 32);
  // column blocks: about two warp units per warp of a one-CTA-per-SM grid,
  // blocks of at least 128 columns
  const long ng = (n + 31) / 32;
  const long warps = (long)c->plan.sms * 32;
  long ncb = (2 * warps + ng / 2) / ng;
  ncb = std::max(1L, std::min(ncb, (long)((n + 127) / 128)));
  op.cbw = (int)((n + ncb - 1) / ncb);
  op.ncb = (int)((n + op.cbw - 1) / op.cbw);
  const size_t na = (size_t)op.lda * (size_t)n, np = (size_t)op.ncb * (size_t)n;
  if (cudaMalloc(&c->vpool, (na + 2 * (np + kGuardWords)) * sizeof(double)) != cudaSuccess)
    return fail(set_err(c, PRCG_ERR_OOM, "matrix allocation failed"));
  if ((rc = add_guard(c, c->vpool + na + np, kGuardWords)) != PRCG_OK) return fail(rc);
  if ((rc = add_guard(c, c->vpool + na + 2 * np + kGuardWords, kGuardWords)) != PRCG_OK)
    return fail(rc);
  if ((rc = wait_user(c)) != PRCG_OK) return fail(rc);
  if (cudaMemcpy2DAsync(c->vpool, (size_t)op.lda * sizeof(double), A, (size_t)n * sizeof(double),
                        (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDefault,
                        c->cs) != cudaSuccess)
    return fail(cuda_err(c, cudaGetLastError(), "copy of A"));
  op.da = c->vpool;
  op.dpart[0] = c->vpool + na;
  op.dpart[1] = c->vpool + na + np + kGuardWords;
  c->precond = precond;
  c->plan.pc.kind = PC_NONE;
  if (precond == PRCG_PRECOND_JACOBI) {
    k_dense_jacobi<<<c->plan.sms * 4, 256, 0, c->cs>>>(op.da, (int)n, op.lda,
                                                       const_cast<double*>(c->plan.pc.d), c->dbad);
    if ((rc = check_bad(c, "Jacobi needs a positive diagonal")) != PRCG_OK) return fail(rc);
    c->plan.pc.kind = PC_VEC;
  }
  c->launch = launcher_for(op.kind, c->plan.pc.kind);
  if (!c->launch) return fail(set_err(c, PRCG_ERR_UNSUPPORTED, "operator not built"));
  *out = c;
  return PRCG_OK;
}

int prcg_solve(prcg_ctx* c, int variant, const double* b, double* x, double tol, int maxit,
               double* residual_history, int* iters_out, double* final_true_relres_out) {
  if (!c) return set_err(nullptr, PRCG_ERR_INVALID, "ctx is NULL");
  if (!b || !x) return set_err(c, PRCG_ERR_INVALID, "b or x is NULL");
  if (!(tol >= 0.0) || maxit < 0) return set_err(c, PRCG_ERR_INVALID, "tol < 0 or maxit < 0");
  if (variant < 0 || variant > V_PIPE_NR) return set_err(c, PRCG_ERR_INVALID, "unknown variant");
  const int n = c->n;
  int rc;
  if (c->hist_cap < maxit + 1) {
    if (c->hist) cudaFree(c->hist);
    c->hist = nullptr;
    c->hist_cap = 0;
    CK(cudaMalloc(&c->hist, (size_t)(maxit + 1) * sizeof(double)));
    c->hist_cap = maxit + 1;
  }
  // small and medium systems: the whole solve as one persistent cooperative
  // launch.  Dense matrices only while A is about L2-sized: beyond that the
  // product dominates the iteration, and the stand-alone product kernel
  // (8 CTAs of 256 threads per SM) outruns the persistent kernel's in-kernel
  // product (one 1024-thread CTA per SM) by ~11 % at n = 10752.
  const int persist_max =
      c->plan.op.kind == OP_DENSE ? std::min(c->persist_max, kDensePersistMax) : c->persist_max;
  // every variant but the two no-recompute ablations has a persistent form
  const bool ablation = variant == V_PR_NR || variant == V_PIPE_NR;
  const bool persist = n <= persist_max && !ablation;
  bool graph = !persist && c->use_graph;
  if (graph && build_graph(c, variant) != PRCG_OK) graph = false;  // fall back to the host loop
  const int chunk = graph ? c->graphs[variant].chunk : chunk_for(c);
  if ((rc = wait_user(c)) != PRCG_OK) return rc;
  if ((rc = copy_in(c, (void*)c->plan.v.b, b, (size_t)n * sizeof(double))) != PRCG_OK) return rc;
  if ((rc = copy_in(c, c->plan.v.x, x, (size_t)n * sizeof(double))) != PRCG_OK) return rc;
  DevState& h = *c->hS;
  memset(&h, 0, sizeof h);
  h.tol = tol;
  h.tol2 = tol * tol;
  h.hist = c->hist;
  c->trace_slots = 0;
  if (c->trace_on) {
    if (c->trace_cap < maxit + 2) {
      if (c->trace) cudaFree(c->trace);
      c->trace = nullptr;
      c->trace_cap = 0;
      CK(cudaMalloc(&c->trace, (size_t)(maxit + 2) * kTraceFields * sizeof(double)));
      c->trace_cap = maxit + 2;
    }
    // all-ones bytes: every unset field reads as NaN
    CK(cudaMemsetAsync(c->trace, 0xFF, (size_t)(maxit + 2) * kTraceFields * sizeof(double), c->cs));
    h.trace = c->trace;
  }
  h.maxit = maxit;
  h.maxbodies = maxit / chunk + 3;
  h.status = kRunning;
  h.carry_nu = variant == V_PR_NR ? 1 : 0;
  h.pf_allow = fixed_p_allowed();
  CK(cudaMemcpyAsync(c->S, &h, sizeof h, cudaMemcpyHostToDevice, c->cs));
  CK(cudaEventRecord(c->ev_start, c->cs));
  bool persisted = false;
  if (persist) {
    if (!c->inject_once) {
      c->hgb = GridBar{};
      c->hgb.spin_limit = kBarrierSpinLimit;
      c->hgb.skip_cta = -1;
      c->hgb.skip_epoch = -1;
    }
    c->inject_once = false;
    CK(cudaMemcpyAsync(c->gb, &c->hgb, sizeof(GridBar), cudaMemcpyHostToDevice, c->cs));
    CK(cudaEventRecord(c->ev_init, c->cs));
    cudaError_t e = c->launch(c->plan, PH_PERSIST, variant, 0, 0, c->cs);
    if (e == cudaSuccess) {
      persisted = true;
      CK(cudaEventRecord(c->ev_loop, c->cs));
    } else {
      cudaGetLastError();   // not launchable cooperatively here: use the graph path
      graph = c->use_graph && build_graph(c, variant) == PRCG_OK;
    }
  }
  if (!persisted) {
    if (graph) {
      CK(cudaGraphLaunch(c->graphs[variant].exec, c->cs));
    } else {
      c->host_loop_launches = 0;
      if ((rc = run_host_loop(c, variant, maxit)) != PRCG_OK) return rc;
    }
  }
  CK(cudaMemcpyAsync(&h, c->S, sizeof h, cudaMemcpyDeviceToHost, c->cs));
  CK(cudaStreamSynchronize(c->cs));
  c->last_pf_sweeps = h.pf_sweeps;
  const int K = h.k;
  {
    const int64_t per_iter = iter_launches(variant) + product_prepasses(c);
    int64_t launches = init_launches(variant) + 2 * product_prepasses(c);
    if (persisted)
      launches = 1;
    else if (graph)
      launches += (int64_t)h.bodies * (chunk * per_iter + 1);
    else
      launches += c->host_loop_launches;
    if (final_true_relres_out) launches += 1 + product_prepasses(c);
    c->last_launches = launches;
  }
  const int status = h.status;
  if (status == kRunning) return set_err(c, PRCG_ERR_CUDA, "device loop ended without a status");
  if (status < 0)
    return set_err(c, status,
                   "device loop did not finish: a bounded wait (grid barrier or copy) expired "
                   "or the loop-body limit was reached");
  if (h.zero_rhs) CK(cudaMemsetAsync(c->plan.v.x, 0, (size_t)n * sizeof(double), c->cs));
  CK(cudaMemcpyAsync(x, c->plan.v.x, (size_t)n * sizeof(double), cudaMemcpyDefault, c->cs));
  if (residual_history) {
    // the device recorded rho_k = ||r_k||^2: convert to ||r_k|| / ||b||
    std::vector<double> hh(K + 1);
    CK(cudaMemcpyAsync(hh.data(), c->hist, (size_t)(K + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                       c->cs));
    CK(cudaStreamSynchronize(c->cs));
    const double bn = sqrt(h.bnorm2);
    for (int k = 0; k <= K; ++k) hh[k] = bn > 0.0 ? sqrt(hh[k]) / bn : 0.0;
    CK(cudaMemcpyAsync(residual_history, hh.data(), (size_t)(K + 1) * sizeof(double),
                       cudaMemcpyDefault, c->cs));
    CK(cudaStreamSynchronize(c->cs));
  }
  if (final_true_relres_out) {
    if (h.zero_rhs) {
      *final_true_relres_out = 0.0;
    } else {
      if ((rc = (c->launch(c->plan, PH_TRUE_RES, variant, 0, 0, c->cs) == cudaSuccess
                     ? PRCG_OK
                     : cuda_err(c, cudaGetLastError(), "true residual"))) != PRCG_OK)
        return rc;
      DevState h2;
      CK(cudaMemcpyAsync(&h2, c->S, sizeof h2, cudaMemcpyDeviceToHost, c->cs));
      CK(cudaStreamSynchronize(c->cs));
      *final_true_relres_out = sqrt(h2.eta) / sqrt(h2.nu_pred);
    }
  }
  CK(cudaStreamSynchronize(c->cs));
  float ti = 0.f, tl = 0.f;
  if (cudaEventElapsedTime(&ti, c->ev_start, c->ev_init) != cudaSuccess) ti = -1.f;
  if (cudaEventElapsedTime(&tl, c->ev_init, c->ev_loop) != cudaSuccess) tl = -1.f;
  cudaGetLastError();
  c->t_init = ti;
  c->t_loop = tl;
  c->last_iters = K;
  if (c->trace_on) c->trace_slots = K + 1;
  if (iters_out) *iters_out = K;
  return status;
}

int prcg_time_sweeps(prcg_ctx* c, int variant, int reps, float* ms_per_sweep, int* nsweeps) {
  if (!c || !ms_per_sweep || !nsweeps || reps < 1) return set_err(c, PRCG_ERR_INVALID, "bad argument");
  if (variant < 0 || variant > 6)
    return set_err(c, PRCG_ERR_UNSUPPORTED, "variant not timed (unknown or an ablation)");
  int phases[3];
  int np = 0;
  if (variant == V_HS) {
    phases[0] = PH_HS_A; phases[1] = PH_HS_B; phases[2] = PH_HS_C; np = 3;
  } else if (variant == V_PR || variant == V_M) {
    phases[0] = PH_PR_A; phases[1] = PH_PR_B; np = 2;
  } else if (variant == V_CGCG) {
    phases[0] = PH_CG_A; phases[1] = PH_CG_B; np = 2;
  } else if (variant == V_GV) {
    phases[0] = PH_GV; np = 1;
  } else {
    phases[0] = PH_PIPE; np = 1;
  }
  cudaEvent_t ev[4];
  for (int q = 0; q <= np; ++q) CK(cudaEventCreate(&ev[q]));
  // a fixed unstructured b, x_0 = 0.  (With b = 1 the iterates of a
  // constant stencil stay exactly zero away from the boundary for the first
  // iterations, rows whose neighbour sums take the all-zero branch.)
  int rc = PRCG_OK;
  DevState& h = *c->hS;
  memset(&h, 0, sizeof h);
  h.tol = 0.0;
  h.maxit = 1 << 30;
  h.status = kRunning;
  h.profile = 1;
  h.maxbodies = 1 << 30;
  h.pf_allow = fixed_p_allowed();
  double tsum[3] = {0, 0, 0};
  cudaError_t e = cudaMemsetAsync(c->plan.v.x, 0, (size_t)c->n * sizeof(double), c->cs);
  if (e == cudaSuccess) {
    k_fill_hashed<<<c->plan.sms * 4, 256, 0, c->cs>>>(const_cast<double*>(c->plan.v.b), c->n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->S, &h, sizeof h, cudaMemcpyHostToDevice, c->cs);
  if (e != cudaSuccess) rc = cuda_err(c, e, "time_sweeps setup");
  if (rc == PRCG_OK) rc = launch_init(c, variant, c->cs);
  // two untimed iterations first: from the third on, the product sweeps of
  // a constant stencil read their block fixed-point copies, as in a solve
  const int warm = 2;
  for (int it = 0; rc == PRCG_OK && it < warm; ++it)
    for (int q = 0; q < np && rc == PRCG_OK; ++q) {
      e = c->launch(c->plan, phases[q], variant, it & 1, (it + 1) & 1, c->cs);
      if (e != cudaSuccess) rc = cuda_err(c, e, "time_sweeps launch");
    }
  for (int it = warm; rc == PRCG_OK && it < warm + reps; ++it) {
    const int qr = it & 1, qw = (it + 1) & 1;
    for (int q = 0; q < np && rc == PRCG_OK; ++q) {
      e = cudaEventRecord(ev[q], c->cs);
      if (e == cudaSuccess) e = c->launch(c->plan, phases[q], variant, qr, qw, c->cs);
      if (e == cudaSuccess) e = cudaEventRecord(ev[q + 1], c->cs);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[q + 1]);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
      if (e != cudaSuccess) rc = cuda_err(c, e, "time_sweeps launch");
      tsum[q] += ms;
    }
  }
  for (int q = 0; q <= np; ++q) cudaEventDestroy(ev[q]);
  if (rc != PRCG_OK) return rc;
  for (int q = 0; q < np; ++q) ms_per_sweep[q] = (float)(tsum[q] / reps);
  *nsweeps = np;
  return PRCG_OK;
}

int prcg_solve_f32_refined(prcg_ctx* c, const double* b, double* x, double tol, int max_outer,
                           double inner_tol, int inner_maxit, int* outer_out, int* inner_total_out,
                           double* final_true_relres_out, double* outer_history) {
  if (!c) return set_err(nullptr, PRCG_ERR_INVALID, "ctx is NULL");
  if (!b || !x) return set_err(c, PRCG_ERR_INVALID, "b or x is NULL");
  if (!(tol >= 0.0) || max_outer < 0 || !(inner_tol > 0.0) || inner_tol >= 1.0 || inner_maxit < 1)
    return set_err(c, PRCG_ERR_INVALID, "bad tolerance or iteration limit");
  const int n = c->n;
  if (c->plan.op.kind == OP_CSR)
    return set_err(c, PRCG_ERR_UNSUPPORTED, "mixed precision needs the SELL-32 layout");
  if (c->plan.op.kind == OP_DENSE)
    return set_err(c, PRCG_ERR_UNSUPPORTED, "mixed precision is not built for dense matrices");
  if (!c->pool32) {
    // six FP32 vectors, each followed by a guard band (from its rounding up
    // to 64 entries, 64 more floats)
    const size_t nr32 = ((size_t)n + 63) / 64 * 64, st32 = nr32 + 2 * kGuardWords;
    CK(cudaMalloc(&c->pool32, 6 * st32 * sizeof(float)));
    CK(cudaMalloc(&c->S2, sizeof(DevState)));
    float* q = c->pool32;
    for (int v = 0; v < 6; ++v) {
      const int grc = add_guard(c, q + v * st32 + nr32, kGuardWords);
      if (grc != PRCG_OK) return grc;
    }
    Vecs32& W = c->plan.w;
    W.r = q; W.rt = q + st32; W.p = q + 2 * st32; W.s = q + 3 * st32;
    W.d = q + 4 * st32; W.rhs = q + 5 * st32;
    c->plan.S2 = c->S2;
    if (c->plan.op.kind == OP_SELL) {
      const int nslices = (n + 31) / 32;
      int total = 0;
      CK(cudaMemcpy(&total, c->plan.op.sptr + nslices, sizeof(int), cudaMemcpyDeviceToHost));
      CK(cudaMalloc(&c->sval32, ((size_t)total + 4) * sizeof(float)));
      k_to_f32<<<c->plan.sms * 8, 256, 0, c->cs>>>(c->plan.op.sval, c->sval32, total);
      CK(cudaGetLastError());
      c->plan.op.sval32 = c->sval32;
    }
  }
  int rc;
  if ((rc = wait_user(c)) != PRCG_OK) return rc;
  if ((rc = copy_in(c, (void*)c->plan.v.b, b, (size_t)n * sizeof(double))) != PRCG_OK) return rc;
  if ((rc = copy_in(c, c->plan.v.x, x, (size_t)n * sizeof(double))) != PRCG_OK) return rc;
  bool graph = c->use_graph;
  if (graph && build_graph(c, kMixedGraph) != PRCG_OK) graph = false;
  CK(cudaMemsetAsync(c->S, 0, sizeof(DevState), c->cs));
  CK(cudaEventRecord(c->ev_start, c->cs));
  int status = PRCG_NOT_CONVERGED, outer = 0, inner_total = 0;
  double rel = 0.0, prev = INFINITY;
  int64_t launches = 0;
  const int chunk = 16;
  for (;;) {
    CK(c->launch(c->plan, PH_MX_RESID, 0, 0, 0, c->cs));
    ++launches;
    DevState h;
    CK(cudaMemcpyAsync(&h, c->S, sizeof h, cudaMemcpyDeviceToHost, c->cs));
    CK(cudaStreamSynchronize(c->cs));
    const double tn = sqrt(h.eta), bn = sqrt(h.nu_pred);
    if (bn == 0.0) {
      CK(cudaMemsetAsync(c->plan.v.x, 0, (size_t)n * sizeof(double), c->cs));
      rel = 0.0;
      status = PRCG_OK;
      if (outer_history) outer_history[outer] = 0.0;
      break;
    }
    rel = tn / bn;
    if (outer_history) outer_history[outer] = rel;
    if (rel <= tol) { status = PRCG_OK; break; }
    if (outer >= max_outer || !(rel < prev)) { status = PRCG_NOT_CONVERGED; break; }
    prev = rel;
    // inner FP32 PR-CG on A d = t / ||t||, to inner_tol -- or, when less
    // suffices to reach tol, to a quarter of the remaining reduction
    DevState& hs = *c->hS;
    memset(&hs, 0, sizeof hs);
    hs.tol = std::max(inner_tol, std::min(0.5, 0.25 * tol / rel));
    hs.tol2 = hs.tol * hs.tol;
    hs.maxit = inner_maxit;
    hs.status = kRunning;
    hs.arg = 1.0 / tn;
    const int ichunk = chunk_for(c);
    hs.maxbodies = inner_maxit / ichunk + 3;
    CK(cudaMemcpyAsync(c->S2, &hs, sizeof hs, cudaMemcpyHostToDevice, c->cs));
    DevState h2;
    if (graph) {
      CK(cudaGraphLaunch(c->graphs[kMixedGraph].exec, c->cs));
      CK(cudaMemcpyAsync(&h2, c->S2, sizeof h2, cudaMemcpyDeviceToHost, c->cs));
      CK(cudaStreamSynchronize(c->cs));
      launches += 2 + (int64_t)h2.bodies * (2 * ichunk + 1);
    } else {
      if ((rc = launch_mixed_init(c, c->cs)) != PRCG_OK) return rc;
      launches += 2;
      for (int it = 0; it <= inner_maxit; it += chunk) {
        CK(cudaMemcpyAsync(&h2, c->S2, sizeof h2, cudaMemcpyDeviceToHost, c->cs));
        CK(cudaStreamSynchronize(c->cs));
        if (h2.done) break;
        for (int m = 0; m < chunk; ++m) {
          if ((rc = launch_mixed_iter(c, c->cs)) != PRCG_OK) return rc;
          launches += 2;
        }
      }
      CK(cudaMemcpyAsync(&h2, c->S2, sizeof h2, cudaMemcpyDeviceToHost, c->cs));
      CK(cudaStreamSynchronize(c->cs));
    }
    if (h2.status < 0) return set_err(c, h2.status, "inner loop exceeded its iteration limit");
    inner_total += h2.k;
    if (h2.k == 0) { status = PRCG_BREAKDOWN; break; }
    c->plan.arg = tn;
    CK(c->launch(c->plan, PH_MX_UPDATE, 0, 0, 0, c->cs));
    ++launches;
    ++outer;
  }
  CK(cudaEventRecord(c->ev_loop, c->cs));
  CK(cudaMemcpyAsync(x, c->plan.v.x, (size_t)n * sizeof(double), cudaMemcpyDefault, c->cs));
  CK(cudaStreamSynchronize(c->cs));
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->ev_start, c->ev_loop) != cudaSuccess) ms = -1.f;
  cudaGetLastError();
  c->t_init = 0.f;
  c->t_loop = ms;
  c->last_iters = inner_total;
  c->last_launches = launches;
  if (outer_out) *outer_out = outer;
  if (inner_total_out) *inner_total_out = inner_total;
  if (final_true_relres_out) *final_true_relres_out = rel;
  return status;
}

int prcg_update_faces(prcg_ctx* c, const double* face_coeff, double diag_shift) {
  if (!c || !face_coeff) return set_err(c, PRCG_ERR_INVALID, "NULL argument");
  OpDesc& op = c->plan.op;
  if (op.kind != OP_VC2 && op.kind != OP_VC3)
    return set_err(c, PRCG_ERR_INVALID, "context has no face coefficients");
  if (!(diag_shift >= 0.0) || !std::isfinite(diag_shift))
    return set_err(c, PRCG_ERR_INVALID, "diag_shift must be finite and >= 0");
  const int dim = op.kind == OP_VC2 ? 2 : 3;
  const size_t nf = (size_t)op.nz * op.ny * (op.nx + 1) + (size_t)op.nz * (op.ny + 1) * op.nx +
                    (dim == 3 ? (size_t)(op.nz + 1) * op.ny * op.nx : 0);
  int rc;
  if ((rc = wait_user(c)) != PRCG_OK) return rc;
  const size_t nfx = (size_t)op.nz * op.ny * (op.nx + 1), nfy = (size_t)op.nz * (op.ny + 1) * op.nx;
  if ((rc = copy_faces(c, op, face_coeff, nfx, nfy, nf - nfx - nfy)) != PRCG_OK) return rc;
  double* d = c->plan.pc.kind == PC_VEC ? const_cast<double*>(c->plan.pc.d) : nullptr;
  k_vc_diag<<<c->plan.sms * 4, 256, 0, c->cs>>>(dim, op.nx, op.ny, op.nz, op.fx, op.fy, op.fz,
                                               diag_shift, const_cast<double*>(op.adiag), d, c->dbad);
  return check_bad(c, "Jacobi needs a positive diagonal");
}

int prcg_grad_faces(prcg_ctx* c, const double* lambda, const double* x, double* grad_faces) {
  if (!c || !lambda || !x || !grad_faces) return set_err(c, PRCG_ERR_INVALID, "NULL argument");
  const OpDesc& op = c->plan.op;
  if (op.kind != OP_VC2 && op.kind != OP_VC3)
    return set_err(c, PRCG_ERR_INVALID, "context has no face coefficients");
  const int dim = op.kind == OP_VC2 ? 2 : 3;
  const size_t n = (size_t)c->n;
  const size_t nf = (size_t)op.nz * op.ny * (op.nx + 1) + (size_t)op.nz * (op.ny + 1) * op.nx +
                    (dim == 3 ? (size_t)(op.nz + 1) * op.ny * op.nx : 0);
  int rc;
  if ((rc = wait_user(c)) != PRCG_OK) return rc;
  // lambda -> t, x -> the x buffer; the gradient is formed in the scratch s buffers
  if ((rc = copy_in(c, c->plan.v.t, lambda, n * sizeof(double))) != PRCG_OK) return rc;
  if ((rc = copy_in(c, c->plan.v.x, x, n * sizeof(double))) != PRCG_OK) return rc;
  if (!c->gscratch) {
    CK(cudaMalloc(&c->gscratch, (nf + kGuardWords) * sizeof(double)));
    if ((rc = add_guard(c, c->gscratch + nf, kGuardWords)) != PRCG_OK) return rc;
  }
  double* g = c->gscratch;
  k_grad_faces<<<c->plan.sms * 8, 256, 0, c->cs>>>(dim, op.nx, op.ny, op.nz, c->plan.v.t,
                                                  c->plan.v.x, g);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(grad_faces, g, nf * sizeof(double), cudaMemcpyDefault, c->cs));
  CK(cudaStreamSynchronize(c->cs));
  return PRCG_OK;
}

int prcg_grad_csr_values(prcg_ctx* c, const double* lambda, const double* x, double* grad_vals) {
  if (!c || !lambda || !x || !grad_vals) return set_err(c, PRCG_ERR_INVALID, "NULL argument");
  const OpDesc& op = c->plan.op;
  if (!op.rp) return set_err(c, PRCG_ERR_INVALID, "context is not a CSR matrix");
  const size_t n = (size_t)c->n;
  int nnz = 0;
  CK(cudaMemcpy(&nnz, op.rp + n, sizeof(int), cudaMemcpyDeviceToHost));
  int rc;
  if ((rc = wait_user(c)) != PRCG_OK) return rc;
  if ((rc = copy_in(c, c->plan.v.t, lambda, n * sizeof(double))) != PRCG_OK) return rc;
  if ((rc = copy_in(c, c->plan.v.x, x, n * sizeof(double))) != PRCG_OK) return rc;
  double* g = nullptr;
  const bool direct = [&] {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, grad_vals) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  }();
  if (direct) {
    g = grad_vals;
  } else {
    CK(cudaMalloc(&g, (size_t)nnz * sizeof(double)));
  }
  k_grad_csr<<<c->plan.sms * 4, 256, 0, c->cs>>>(op.rp, op.ci, (int)n, c->plan.v.t, c->plan.v.x, g);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !direct)
    e = cudaMemcpyAsync(grad_vals, g, (size_t)nnz * sizeof(double), cudaMemcpyDeviceToHost, c->cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->cs);
  if (!direct) cudaFree(g);
  if (e != cudaSuccess) return cuda_err(c, e, "CSR value gradient");
  return PRCG_OK;
}

int prcg_last_timing(const prcg_ctx* c, float* init_ms, float* loop_ms, int* iters) {
  if (!c) return PRCG_ERR_INVALID;
  if (init_ms) *init_ms = c->t_init;
  if (loop_ms) *loop_ms = c->t_loop;
  if (iters) *iters = c->last_iters;
  return PRCG_OK;
}

int prcg_last_fixed_sweeps(const prcg_ctx* c, int64_t* sweeps) {
  if (!c || !sweeps) return PRCG_ERR_INVALID;
  *sweeps = c->last_pf_sweeps;
  return PRCG_OK;
}

int prcg_last_launches(const prcg_ctx* c, int64_t* kernels) {
  if (!c || !kernels) return PRCG_ERR_INVALID;
  *kernels = c->last_launches;
  return PRCG_OK;
}

int prcg_jacobi_form(const prcg_ctx* c) {
  if (!c) return PRCG_ERR_INVALID;
  return c->plan.pc.kind == PC_SCALAR ? 1 : c->plan.pc.kind == PC_VEC ? 2 : 0;
}

int prcg_int_diagonal(const prcg_ctx* c) {
  if (!c) return PRCG_ERR_INVALID;
  const int k = c->plan.op.kind;
  return (k == OP_ST2 || k == OP_ST3) ? c->plan.op.cint : 0;
}

int prcg_destroy(prcg_ctx* c) {
  if (!c) return PRCG_OK;
  if (c->cs) cudaStreamSynchronize(c->cs);
  destroy_graphs(c);
  if (c->pool) cudaFree(c->pool);
  if (c->ipool) cudaFree(c->ipool);
  if (c->vpool) cudaFree(c->vpool);
  if (c->sell_i) cudaFree(c->sell_i);
  if (c->pool32) cudaFree(c->pool32);
  if (c->sval32) cudaFree(c->sval32);
  if (c->S2) cudaFree(c->S2);
  if (c->gb) cudaFree(c->gb);
  if (c->sell_v) cudaFree(c->sell_v);
  if (c->partials) cudaFree(c->partials);
  if (c->S) cudaFree(c->S);
  if (c->hS) cudaFreeHost(c->hS);
  if (c->hist) cudaFree(c->hist);
  if (c->trace) cudaFree(c->trace);
  if (c->dguard) cudaFree(c->dguard);
  if (c->gscratch) cudaFree(c->gscratch);
  if (c->dbad) cudaFree(c->dbad);
  if (c->ev_user) cudaEventDestroy(c->ev_user);
  if (c->ev_start) cudaEventDestroy(c->ev_start);
  if (c->ev_init) cudaEventDestroy(c->ev_init);
  if (c->ev_loop) cudaEventDestroy(c->ev_loop);
  if (c->bs) cudaStreamDestroy(c->bs);
  if (c->cs) cudaStreamDestroy(c->cs);
  delete c;
  return PRCG_OK;
}

const char* prcg_last_error(const prcg_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

int64_t prcg_n(const prcg_ctx* c) { return c ? (int64_t)c->n : -1; }

int prcg_inject_barrier_skip(prcg_ctx* c, int cta, int barrier, int64_t spin_limit) {
  if (!c) return set_err(nullptr, PRCG_ERR_INVALID, "ctx is NULL");
  if (cta < 0 || barrier < 0 || spin_limit < 1024)
    return set_err(c, PRCG_ERR_INVALID, "bad injection");
  c->hgb = GridBar{};
  c->hgb.spin_limit = spin_limit;
  c->hgb.skip_cta = cta;
  c->hgb.skip_epoch = barrier;
  c->inject_once = true;
  return PRCG_OK;
}

int prcg_check_guards(prcg_ctx* c, int64_t* corrupted_out) {
  if (!c || !corrupted_out) return set_err(c, PRCG_ERR_INVALID, "NULL argument");
  CK(cudaMemsetAsync(c->dguard, 0, sizeof(unsigned long long), c->cs));
  for (const auto& g : c->guards)
    k_guard_count<<<1, 256, 0, c->cs>>>(static_cast<const unsigned long long*>(g.first), g.second,
                                        c->dguard);
  CK(cudaGetLastError());
  unsigned long long bad = 0;
  CK(cudaMemcpyAsync(&bad, c->dguard, sizeof bad, cudaMemcpyDeviceToHost, c->cs));
  CK(cudaStreamSynchronize(c->cs));
  *corrupted_out = (int64_t)bad;
  return PRCG_OK;
}

int prcg_test_neighbour_sum(int terms, const double* v, int64_t count, double* out) {
  prcg_ctx* c = nullptr;   // no context: errors go to prcg_last_error(NULL)
  if ((terms != 4 && terms != 6) || count < 0 || (count > 0 && (!v || !out)))
    return set_err(c, PRCG_ERR_INVALID, "terms must be 4 or 6, count >= 0, v and out non-NULL");
  if (count == 0) return PRCG_OK;
  double* dv = nullptr;
  double* dout = nullptr;
  const size_t bin = (size_t)count * terms * sizeof(double), bout = (size_t)count * sizeof(double);
  cudaError_t e = cudaMalloc(&dv, bin);
  if (e == cudaSuccess) e = cudaMalloc(&dout, bout);
  if (e == cudaSuccess) e = cudaMemcpy(dv, v, bin, cudaMemcpyDefault);
  if (e == cudaSuccess) {
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
    if (terms == 4)
      k_test_neighbour_sum<4><<<(int)blocks, 256>>>(dv, count, dout);
    else
      k_test_neighbour_sum<6><<<(int)blocks, 256>>>(dv, count, dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, bout, cudaMemcpyDefault);
  if (dv) cudaFree(dv);
  if (dout) cudaFree(dout);
  return e == cudaSuccess ? PRCG_OK : cuda_err(c, e, "neighbour sum test");
}

int prcg_trace_enable(prcg_ctx* c, int on) {
  if (!c) return set_err(nullptr, PRCG_ERR_INVALID, "ctx is NULL");
  c->trace_on = on != 0;
  c->trace_slots = 0;
  return PRCG_OK;
}

int prcg_trace_get(prcg_ctx* c, double* out, int slots) {
  if (!c) return set_err(nullptr, PRCG_ERR_INVALID, "ctx is NULL");
  if (!out || slots < 0) return set_err(c, PRCG_ERR_INVALID, "bad argument");
  const int m = std::min(slots, c->trace_slots);
  if (m > 0) {
    CK(cudaMemcpyAsync(out, c->trace, (size_t)m * kTraceFields * sizeof(double), cudaMemcpyDefault,
                       c->cs));
    CK(cudaStreamSynchronize(c->cs));
  }
  return m;
}

int prcg_error_anorm(prcg_ctx* c, const double* x_star, const double* x, double* err_out) {
  if (!c) return set_err(nullptr, PRCG_ERR_INVALID, "ctx is NULL");
  if (!x_star || !x || !err_out) return set_err(c, PRCG_ERR_INVALID, "NULL argument");
  const size_t bytes = (size_t)c->n * sizeof(double);
  int rc;
  if ((rc = wait_user(c)) != PRCG_OK) return rc;
  if ((rc = copy_in(c, c->plan.v.t, x_star, bytes)) != PRCG_OK) return rc;
  if ((rc = copy_in(c, c->plan.v.w[1], x, bytes)) != PRCG_OK) return rc;
  const cudaError_t e = c->launch(c->plan, PH_ANORM, V_PR, 0, 0, c->cs);
  if (e != cudaSuccess) return cuda_err(c, e, "A-norm error");
  DevState h;
  CK(cudaMemcpyAsync(&h, c->S, sizeof h, cudaMemcpyDeviceToHost, c->cs));
  CK(cudaStreamSynchronize(c->cs));
  *err_out = sqrt(h.eta > 0.0 ? h.eta : 0.0);
  return PRCG_OK;
}

}  // extern "C"
