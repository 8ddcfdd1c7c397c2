// Batched PR-CG: many independent 2D 5-point (shifted) stencil systems of
// uneven size solved by one persistent kernel launch.
//
// Every thread-block cluster is a solver: its leader CTA takes the next
// system from a device work queue (systems ordered by estimated cost,
// largest first), and the cluster runs Algorithm 2 on it -- sweep A (x, r,
// r~, p and the partial nu, <r, r>), a cluster barrier, sweep B (s = A p and
// mu, sigma, gamma) and one cluster-wide reduction through distributed shared
// memory -- until the system converges, then takes the next one.  The
// reduction adds the CTA partials in rank order in every CTA, so all CTAs
// of a cluster hold bitwise-identical scalars and take identical decisions;
// the only synchronisation is the hardware cluster barrier (no CTA ever
// spins on memory).  Cluster size and CTA size are launch parameters chosen
// by the autotuner (paper_1905_01549_gb300/autotune.py).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/prcg.h"
#include "prcg_isum.cuh"
#include "prcg_reduce.cuh"

namespace cg = cooperative_groups;

namespace {

struct BatchSys {
  long long off;  // first row in the concatenated vectors
  int nx, ny;
  double cdiag;   // 4 + shift
  double d;       // Jacobi 1 / cdiag, or 1
  prcg::FastDiv divx;   // division by nx
};

constexpr int kMaxThreads = 1024;

// Cluster-wide sum followed by the scalar step.  CTA totals go to a
// double-buffered shared slot and, after one cluster barrier, warp 0 of every
// CTA gathers the ranks' slots (lane r takes rank r) and adds them in a fixed
// tree, so all CTAs of the cluster form bitwise-identical totals.  Warp 0
// alone then runs `step(tot, bc)`, which leaves its results in the shared
// array bc (lane 0 stores): the FP64 pipe issues two lanes per clock per SM
// here, so neither the rank sums nor the divisions of the scalar step are
// repeated in every warp.  Ranks are at most 32 (portable clusters are <= 8,
// non-portable <= 16).
template <int NV, class Step>
__device__ __forceinline__ void cluster_sum(double (&v)[NV], double* sm, double* slots, int& parity,
                                            cg::cluster_group& cl, bool warp_active, Step&& step) {
  prcg::block_sum<NV>(v, sm, warp_active);
  double* mine = slots + parity * 8;
  if (threadIdx.x == 0)
#pragma unroll
    for (int m = 0; m < NV; ++m) mine[m] = v[m];
  cl.sync();
  if (threadIdx.x < 32) {
    const unsigned lane = threadIdx.x;
    double t[NV];
    const bool has = lane < cl.num_blocks();
    const double* rs = cl.map_shared_rank(mine, has ? lane : 0u);
#pragma unroll
    for (int m = 0; m < NV; ++m) t[m] = has ? rs[m] : 0.0;
    __syncwarp();
    prcg::warp_sum_store<NV>(t, sm, 1);   // totals to sm[0..NV)
    __syncwarp();
    double tot[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) tot[m] = sm[m];
    step(tot);
  }
  __syncthreads();
  parity ^= 1;
}

// The plain FP64 sum of the rare neighbour tuples the fixed-point path
// declines (non-finite or extreme terms).  Out of line, with the terms in
// registers: inlined into this kernel, the branch around the additions was
// turned into predicated FP64 instructions issued on every row (ncu on 128
// systems: 11.7 FP64 instructions per row-iteration instead of 8.7, 62 ms
// instead of 53 ms).
static __device__ __noinline__ double sequential_sum4(double a, double b, double c, double d) {
  return ((a + b) + c) + d;
}

// (A v)_i = cdiag v_i - sum of the existing neighbours; the neighbour sum is
// exact in fixed point on the integer pipes and rounded once
// (prcg_isum.cuh), leaving one FP64 FMA per row.
__device__ __forceinline__ double stencil_row(const BatchSys& q, const double* __restrict__ v,
                                              int i) {
  const int y = prcg::fast_div(q.divx, i), x = i - y * q.nx;
  const double ym = __ldcg(v + (y > 0 ? i - q.nx : i));
  const double xm = __ldcg(v + (x > 0 ? i - 1 : i));
  const double xp = __ldcg(v + (x < q.nx - 1 ? i + 1 : i));
  const double yp = __ldcg(v + (y < q.ny - 1 ? i + q.nx : i));
  const double nb[4] = {y > 0 ? ym : 0.0, x > 0 ? xm : 0.0, x < q.nx - 1 ? xp : 0.0,
                        y < q.ny - 1 ? yp : 0.0};
  double sum;
  if (!prcg::fixed_point_sum<4>(nb, sum)) sum = sequential_sum4(nb[0], nb[1], nb[2], nb[3]);
  return fma(q.cdiag, __ldcg(v + i), -sum);
}

struct BatchArgs {
  const BatchSys* sys;
  const int* order;     // systems by decreasing estimated cost
  int nsys;
  const double* b;
  double* x;
  double* r;
  double* rt;
  double* p;
  double* s;
  double tol;
  int maxit;
  int jacobi;
  int* iters;
  int* status;
  int* queue;
};

// JAC: Jacobi preconditioning (a compile-time choice, so the unpreconditioned
// kernel issues no FP64 instruction for it -- a run-time branch around an FMA
// may be if-converted into a predicated instruction that still issues).
template <bool JAC>
__global__ void __launch_bounds__(kMaxThreads) k_batched_pr(BatchArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const unsigned crank = cl.block_rank();
  const int G = (int)(cl.num_blocks() * blockDim.x);
  const int g0 = (int)(crank * blockDim.x + threadIdx.x);
  __shared__ double sm[5 * 32];
  __shared__ double slots[2 * 8];
  __shared__ double bc[3];      // what warp 0 decided, read by every thread
  __shared__ int bst;           // status decided by warp 0 (-100: running)
  __shared__ int s_next;
  int parity = 0;
  for (;;) {
    if (crank == 0 && threadIdx.x == 0) s_next = atomicAdd(a.queue, 1);
    cl.sync();
    const int qi = *cl.map_shared_rank(&s_next, 0);
    cl.sync();  // the leader's slot is read by all before it is rewritten
    if (qi >= a.nsys) break;
    const int id = a.order[qi];
    const BatchSys q = a.sys[id];
    const int n = q.nx * q.ny;
    const bool wact = g0 - (int)(threadIdx.x & 31) < n;   // this warp owns rows
    const double* b = a.b + q.off;
    double* x = a.x + q.off;
    double* r = a.r + q.off;
    double* rt = a.rt + q.off;
    double* p = a.p + q.off;
    double* s = a.s + q.off;
    const double d = q.d;
    // initialize(): r_0 = b - A x_0, r~_0 = d r_0, p_0 = r~_0
    double i3[3] = {0.0, 0.0, 0.0};
    for (int i = g0; i < n; i += G) {
      const double bi = b[i];
      const double ri = bi - stencil_row(q, x, i);
      const double rti = JAC ? d * ri : ri;
      r[i] = ri;
      rt[i] = rti;
      p[i] = rti;
      i3[0] = fma(rti, ri, i3[0]);
      i3[1] = fma(ri, ri, i3[1]);
      i3[2] = fma(bi, bi, i3[2]);
    }
    // bc = {nu_0, tol^2 ||b||^2 (||r||^2 <= that stops), b == 0, status}
    cluster_sum<3>(i3, sm, slots, parity, cl, wact, [&](const double* t) {
      const double stop2 = a.tol * a.tol * t[2];
      int st = -100;
      if (t[2] == 0.0 || t[1] <= stop2)
        st = 0;
      else if (a.maxit == 0)
        st = 1;
      if (threadIdx.x == 0) {
        bc[0] = t[0];
        bc[1] = stop2;
        bc[2] = t[2] == 0.0 ? 1.0 : 0.0;
        bst = st;
      }
    });
    double nu = bc[0];
    const double stop2 = bc[1];
    int status = bst, K = 0;
    if (bc[2] != 0.0)
      for (int i = g0; i < n; i += G) x[i] = 0.0;
    if (status == -100) {
      // s_0 = A p_0; mu_0, sigma_0, gamma_0 -> alpha_1, beta_1 (Eq. 2.3)
      double j3[3] = {0.0, 0.0, 0.0};
      for (int i = g0; i < n; i += G) {
        const double si = stencil_row(q, p, i);
        s[i] = si;
        j3[0] = fma(p[i], si, j3[0]);
        j3[1] = fma(rt[i], si, j3[1]);
        j3[2] = fma(si, si, j3[2]);
      }
      // the scalar step: alpha_k = nu/mu, nu'_{k+1} = nu - 2 alpha sigma + alpha^2 gamma,
      // beta = nu'/nu; status 2 on breakdown
      auto scalars = [&](double nu_, double mu, double sigma, double gamma) {
        const double alpha = nu_ / mu;
        const double nu_pred = nu_ - 2.0 * alpha * sigma + alpha * alpha * gamma;
        const bool bad = !isfinite(nu_) || !isfinite(mu) || !(mu > 0.0) || nu_ < 0.0 ||
                         !isfinite(nu_pred) || nu_pred < 0.0 || nu_ == 0.0;
        if (threadIdx.x == 0) {
          bc[0] = alpha;
          bc[1] = bad ? 0.0 : nu_pred / nu_;
          bc[2] = nu_;
          bst = bad ? 2 : -100;
        }
      };
      cluster_sum<3>(j3, sm, slots, parity, cl, wact, [&](const double* t) {
        scalars(nu, t[0], t[1], JAC ? d * t[2] : t[2]);
      });
      status = bst;
      double alpha = bc[0], beta = bc[1];
      for (int k = 1; status == -100 && k <= a.maxit; ++k) {
        // sweep A: x_k, r_k, r~_k, p_k
        double a2[2] = {0.0, 0.0};
        for (int i = g0; i < n; i += G) {
          const double si = s[i];
          const double pi = p[i];
          x[i] = fma(alpha, pi, x[i]);
          const double rn = fma(-alpha, si, r[i]);
          r[i] = rn;
          double rtn = rn;
          if (JAC) {
            rtn = fma(-alpha, d * si, rt[i]);
            rt[i] = rtn;
          }
          p[i] = fma(beta, pi, rtn);
          if (JAC) a2[0] = fma(rtn, rn, a2[0]);   // unpreconditioned: nu_k = <r_k, r_k>
          a2[1] = fma(rn, rn, a2[1]);
        }
        cl.sync();  // p_k complete in every CTA before the product
        // sweep B: s_k = A p_k, mu_k, sigma_k, gamma_k
        double a5[5] = {a2[0], a2[1], 0.0, 0.0, 0.0};
        const double* rtv = JAC ? rt : r;
        for (int i = g0; i < n; i += G) {
          const double sn = stencil_row(q, p, i);
          s[i] = sn;
          a5[2] = fma(p[i], sn, a5[2]);
          a5[3] = fma(rtv[i], sn, a5[3]);
          a5[4] = fma(sn, sn, a5[4]);
        }
        // stop on ||r_k||^2 <= tol^2 ||b||^2, else the scalars of iteration k + 1
        cluster_sum<5>(a5, sm, slots, parity, cl, wact, [&](const double* t) {
          if (t[1] <= stop2 || k == a.maxit) {
            if (threadIdx.x == 0) bst = t[1] <= stop2 ? 0 : 1;
          } else {
            scalars(JAC ? t[0] : t[1], t[2], t[3], JAC ? d * t[4] : t[4]);
          }
        });
        K = k;
        status = bst;
        alpha = bc[0];
        beta = bc[1];
      }
    }
    if (crank == 0 && threadIdx.x == 0) {
      a.iters[id] = K;
      a.status[id] = status;
    }
  }
}

// ||b - A x|| / ||b|| per system (one CTA per system, grid-stride over systems).
__global__ void k_batched_true_res(BatchArgs a, double* out) {
  __shared__ double sm[2 * 32];
  for (int id = blockIdx.x; id < a.nsys; id += gridDim.x) {
    const BatchSys q = a.sys[id];
    const int n = q.nx * q.ny;
    double v[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double bi = a.b[q.off + i];
      const double t = bi - stencil_row(q, a.x + q.off, i);
      v[0] = fma(t, t, v[0]);
      v[1] = fma(bi, bi, v[1]);
    }
    prcg::block_sum<2>(v, sm);
    if (threadIdx.x == 0) out[id] = v[1] > 0.0 ? sqrt(v[0]) / sqrt(v[1]) : 0.0;
    __syncthreads();
  }
}

}  // namespace

struct prcg_batch {
  int nsys = 0;
  long long total = 0;
  int precond = 0;
  cudaStream_t user = nullptr, cs = nullptr;
  cudaEvent_t ev_user = nullptr, ev0 = nullptr, ev1 = nullptr;
  BatchSys* d_sys = nullptr;
  int* d_order = nullptr;
  int* d_iters = nullptr;
  int* d_status = nullptr;
  int* d_queue = nullptr;
  double* d_true = nullptr;
  double* pool = nullptr;  // b, x, r, r~, p, s
  int cluster = 1;
  int threads = 256;
  int clusters = 0;
  // Split launch (split > 0): the `split` systems of largest estimated cost
  // run on clusters of cluster x threads, the others on a second,
  // independent persistent launch of cluster2 x threads2 beside it (own work
  // queue, forked and joined inside the same graph); 0: one launch.
  int split = 0;
  int cluster2 = 8;
  int threads2 = 512;
  int clusters2 = 0;
  cudaStream_t cs2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t exec = nullptr;
  double graph_tol = -1.0;   // parameters the instantiated graph was captured with
  int graph_maxit = -1;
  float last_ms = 0.f;
  std::string err;
};

namespace {

int berr(prcg_batch* bt, int code, const std::string& m) {
  if (bt) bt->err = m;
  return code;
}

#define BCK(call)                                                              \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) return berr(bt, PRCG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

BatchArgs args_of(prcg_batch* bt, double tol, int maxit) {
  BatchArgs a;
  a.sys = bt->d_sys;
  a.order = bt->d_order;
  a.nsys = bt->nsys;
  const long long T = bt->total;
  a.b = bt->pool;
  a.x = bt->pool + T;
  a.r = bt->pool + 2 * T;
  a.rt = bt->pool + 3 * T;
  a.p = bt->pool + 4 * T;
  a.s = bt->pool + 5 * T;
  a.tol = tol;
  a.maxit = maxit;
  a.jacobi = bt->precond == PRCG_PRECOND_JACOBI;
  a.iters = bt->d_iters;
  a.status = bt->d_status;
  a.queue = bt->d_queue;
  return a;
}

// One persistent launch of `clusters` clusters of `cluster` CTAs x `threads`;
// `high_priority` asks the block scheduler to place its CTAs first.
cudaError_t launch_batched(const BatchArgs& a, int cluster, int threads, int clusters,
                           bool high_priority, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3(clusters * cluster);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (high_priority) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess) {
      at[1].id = cudaLaunchAttributePriority;
      at[1].val.priority = greatest;
      cfg.numAttrs = 2;
    }
  }
  return a.jacobi ? cudaLaunchKernelEx(&cfg, k_batched_pr<true>, a)
                  : cudaLaunchKernelEx(&cfg, k_batched_pr<false>, a);
}

// Clusters of `cluster` CTAs x `threads` that can be resident at once.
int max_clusters(prcg_batch* bt, int cluster, int threads, int* nc) {
  const bool jac = bt->precond == PRCG_PRECOND_JACOBI;
  const void* kern = jac ? (const void*)k_batched_pr<true> : (const void*)k_batched_pr<false>;
  if (cluster > 8)
    BCK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.gridDim = dim3(cluster);
  cfg.blockDim = dim3(threads);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  *nc = 0;
  BCK(cudaOccupancyMaxActiveClusters(nc, kern, &cfg));
  if (*nc < 1) return berr(bt, PRCG_ERR_UNSUPPORTED, "cluster configuration cannot be resident");
  return PRCG_OK;
}

// Persistent grids: as many clusters as can be resident at once.  For a
// split launch the first launch takes one cluster per large system (at most
// what is resident) and the second what the first leaves free, counted in
// CTA-thread slots, so that both run side by side.
int size_grid(prcg_batch* bt) {
  int nc = 0, rc = max_clusters(bt, bt->cluster, bt->threads, &nc);
  if (rc != PRCG_OK) return rc;
  if (bt->split <= 0) {
    bt->clusters = std::min(nc, bt->nsys);
    bt->clusters2 = 0;
    return PRCG_OK;
  }
  bt->clusters = std::min(nc, bt->split);
  int nc2 = 0;
  if ((rc = max_clusters(bt, bt->cluster2, bt->threads2, &nc2)) != PRCG_OK) return rc;
  const long long slots = (long long)nc2 * bt->cluster2 * bt->threads2;
  const long long used = (long long)bt->clusters * bt->cluster * bt->threads;
  const long long per = (long long)bt->cluster2 * bt->threads2;
  const long long free_clusters = (slots - used) / per;
  bt->clusters2 = (int)std::max(1LL, std::min<long long>(free_clusters, bt->nsys - bt->split));
  return PRCG_OK;
}

void drop_graph(prcg_batch* bt) {
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  bt->exec = nullptr;
}

}  // namespace

extern "C" {

int prcg_batched_create(prcg_batch** out, int nsys, const int32_t* nx, const int32_t* ny,
                        const double* shift, int precond, void* cuda_stream) {
  prcg_batch* bt = nullptr;
  if (!out || nsys < 1 || !nx || !ny || !shift) return PRCG_ERR_INVALID;
  if (precond != PRCG_PRECOND_NONE && precond != PRCG_PRECOND_JACOBI) return PRCG_ERR_INVALID;
  *out = nullptr;
  bt = new prcg_batch();
  bt->nsys = nsys;
  bt->precond = precond;
  bt->user = (cudaStream_t)cuda_stream;
  std::vector<BatchSys> sys(nsys);
  std::vector<double> cost(nsys);
  long long off = 0;
  for (int i = 0; i < nsys; ++i) {
    if (nx[i] < 1 || ny[i] < 1 || (long long)nx[i] * ny[i] >= (1LL << 30) || !(shift[i] >= 0.0) ||
        !std::isfinite(shift[i])) {
      delete bt;
      return PRCG_ERR_INVALID;
    }
    sys[i].off = off;
    sys[i].nx = nx[i];
    sys[i].ny = ny[i];
    sys[i].cdiag = 4.0 + shift[i];
    sys[i].d = precond == PRCG_PRECOND_JACOBI ? 1.0 / sys[i].cdiag : 1.0;
    sys[i].divx = prcg::make_fastdiv(nx[i]);
    const double n = (double)nx[i] * ny[i];
    // work ~ n * sqrt(condition number): lambda_min of the shifted 5-point
    // operator is 2 - 2 cos(pi/(nx+1)) + 2 - 2 cos(pi/(ny+1)) + shift
    const double pi = 3.14159265358979323846;
    const double lmin = 4.0 - 2.0 * cos(pi / (nx[i] + 1)) - 2.0 * cos(pi / (ny[i] + 1)) + shift[i];
    cost[i] = n * sqrt((8.0 + shift[i]) / lmin);
    off += (long long)nx[i] * ny[i];
  }
  bt->total = off;
  std::vector<int> order(nsys);
  for (int i = 0; i < nsys; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  if (cudaStreamCreateWithFlags(&bt->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&bt->cs2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&bt->ev_user, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&bt->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&bt->ev0) != cudaSuccess || cudaEventCreate(&bt->ev1) != cudaSuccess ||
      cudaMalloc(&bt->d_sys, nsys * sizeof(BatchSys)) != cudaSuccess ||
      cudaMalloc(&bt->d_order, nsys * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&bt->d_iters, nsys * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&bt->d_status, nsys * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&bt->d_queue, 2 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&bt->d_true, nsys * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&bt->pool, 6 * (size_t)off * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    prcg_batched_destroy(bt);
    return PRCG_ERR_OOM;
  }
  cudaMemcpy(bt->d_sys, sys.data(), nsys * sizeof(BatchSys), cudaMemcpyHostToDevice);
  cudaMemcpy(bt->d_order, order.data(), nsys * sizeof(int), cudaMemcpyHostToDevice);
  if (size_grid(bt) != PRCG_OK) {
    prcg_batched_destroy(bt);
    return PRCG_ERR_CUDA;
  }
  *out = bt;
  return PRCG_OK;
}

int prcg_batched_configure(prcg_batch* bt, int cluster, int threads) {
  if (!bt) return PRCG_ERR_INVALID;
  if (cluster < 1 || cluster > 16 || (cluster & (cluster - 1)) != 0)
    return berr(bt, PRCG_ERR_INVALID, "cluster must be 1, 2, 4, 8 or 16");
  if (threads < 64 || threads > kMaxThreads || threads % 32 != 0)
    return berr(bt, PRCG_ERR_INVALID, "threads must be a multiple of 32 in [64, 1024]");
  const int oc = bt->cluster, ot = bt->threads, os = bt->split;
  bt->cluster = cluster;
  bt->threads = threads;
  bt->split = 0;
  int rc = size_grid(bt);
  if (rc != PRCG_OK) {
    bt->cluster = oc;
    bt->threads = ot;
    bt->split = os;
    size_grid(bt);
    return rc;
  }
  drop_graph(bt);
  return PRCG_OK;
}

int prcg_batched_configure_split(prcg_batch* bt, int nbig, int cluster_big, int threads_big,
                                 int cluster_rest, int threads_rest) {
  if (!bt) return PRCG_ERR_INVALID;
  if (nbig < 1 || nbig >= bt->nsys)
    return berr(bt, PRCG_ERR_INVALID, "nbig must be in [1, number of systems)");
  for (int c : {cluster_big, cluster_rest})
    if (c < 1 || c > 16 || (c & (c - 1)) != 0)
      return berr(bt, PRCG_ERR_INVALID, "cluster must be 1, 2, 4, 8 or 16");
  for (int t : {threads_big, threads_rest})
    if (t < 64 || t > kMaxThreads || t % 32 != 0)
      return berr(bt, PRCG_ERR_INVALID, "threads must be a multiple of 32 in [64, 1024]");
  const int oc = bt->cluster, ot = bt->threads, os = bt->split, oc2 = bt->cluster2,
            ot2 = bt->threads2;
  bt->cluster = cluster_big;
  bt->threads = threads_big;
  bt->split = nbig;
  bt->cluster2 = cluster_rest;
  bt->threads2 = threads_rest;
  int rc = size_grid(bt);
  if (rc != PRCG_OK) {
    bt->cluster = oc;
    bt->threads = ot;
    bt->split = os;
    bt->cluster2 = oc2;
    bt->threads2 = ot2;
    size_grid(bt);
    return rc;
  }
  drop_graph(bt);
  return PRCG_OK;
}

int prcg_batched_solve(prcg_batch* bt, const double* b, double* x, double tol, int maxit,
                       int32_t* iters_out, int32_t* status_out, double* true_relres_out) {
  if (!bt || !b || !x) return PRCG_ERR_INVALID;
  if (!(tol >= 0.0) || maxit < 0) return berr(bt, PRCG_ERR_INVALID, "tol < 0 or maxit < 0");
  const size_t bytes = (size_t)bt->total * sizeof(double);
  BatchArgs a = args_of(bt, tol, maxit);
  BCK(cudaEventRecord(bt->ev_user, bt->user));
  BCK(cudaStreamWaitEvent(bt->cs, bt->ev_user, 0));
  BCK(cudaMemcpyAsync((void*)a.b, b, bytes, cudaMemcpyDefault, bt->cs));
  BCK(cudaMemcpyAsync(a.x, x, bytes, cudaMemcpyDefault, bt->cs));
  // one graph: reset the work queues, the persistent solver launch (or, for
  // a split, the two launches forked onto two streams and joined again)
  if (bt->exec && (bt->graph_tol != tol || bt->graph_maxit != maxit)) drop_graph(bt);
  if (!bt->exec) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(bt->cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(bt->d_queue, 0, 2 * sizeof(int), bt->cs);
    if (bt->split <= 0) {
      if (e == cudaSuccess)
        e = launch_batched(a, bt->cluster, bt->threads, bt->clusters, false, bt->cs);
    } else {
      BatchArgs big = a, rest = a;
      big.nsys = bt->split;
      rest.order = bt->d_order + bt->split;
      rest.nsys = bt->nsys - bt->split;
      rest.queue = bt->d_queue + 1;
      if (e == cudaSuccess) e = cudaEventRecord(bt->ev_fork, bt->cs);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->cs2, bt->ev_fork, 0);
      if (e == cudaSuccess)
        e = launch_batched(big, bt->cluster, bt->threads, bt->clusters, true, bt->cs);
      if (e == cudaSuccess)
        e = launch_batched(rest, bt->cluster2, bt->threads2, bt->clusters2, false, bt->cs2);
      if (e == cudaSuccess) e = cudaEventRecord(bt->ev_join, bt->cs2);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(bt->cs, bt->ev_join, 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(bt->cs, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return berr(bt, PRCG_ERR_CUDA, std::string("batched graph capture: ") +
                                          cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&bt->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return berr(bt, PRCG_ERR_CUDA, "batched graph instantiate");
    bt->graph_tol = tol;
    bt->graph_maxit = maxit;
  }
  BCK(cudaEventRecord(bt->ev0, bt->cs));
  BCK(cudaGraphLaunch(bt->exec, bt->cs));
  BCK(cudaEventRecord(bt->ev1, bt->cs));
  if (true_relres_out) {
    k_batched_true_res<<<std::min(bt->nsys, 1024), 256, 0, bt->cs>>>(a, bt->d_true);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(true_relres_out, bt->d_true, bt->nsys * sizeof(double), cudaMemcpyDefault,
                        bt->cs));
  }
  BCK(cudaMemcpyAsync(x, a.x, bytes, cudaMemcpyDefault, bt->cs));
  if (iters_out)
    BCK(cudaMemcpyAsync(iters_out, bt->d_iters, bt->nsys * sizeof(int), cudaMemcpyDefault, bt->cs));
  std::vector<int> st(bt->nsys);
  BCK(cudaMemcpyAsync(st.data(), bt->d_status, bt->nsys * sizeof(int), cudaMemcpyDeviceToHost,
                      bt->cs));
  BCK(cudaStreamSynchronize(bt->cs));
  if (status_out) memcpy(status_out, st.data(), bt->nsys * sizeof(int));
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, bt->ev0, bt->ev1) == cudaSuccess) bt->last_ms = ms;
  int worst = PRCG_OK;
  for (int s : st) {
    if (s < 0) return berr(bt, PRCG_ERR_CUDA, "a system finished without a status");
    worst = std::max(worst, s);
  }
  return worst;
}

int prcg_batched_last_ms(const prcg_batch* bt, float* ms) {
  if (!bt || !ms) return PRCG_ERR_INVALID;
  *ms = bt->last_ms;
  return PRCG_OK;
}

int prcg_batched_config(const prcg_batch* bt, int* cluster, int* threads, int* clusters) {
  if (!bt) return PRCG_ERR_INVALID;
  if (cluster) *cluster = bt->cluster;
  if (threads) *threads = bt->threads;
  if (clusters) *clusters = bt->clusters;
  return PRCG_OK;
}

int prcg_batched_split(const prcg_batch* bt, int* nbig, int* cluster_rest, int* threads_rest,
                       int* clusters_rest) {
  if (!bt) return PRCG_ERR_INVALID;
  const bool on = bt->split > 0;
  if (nbig) *nbig = on ? bt->split : 0;
  if (cluster_rest) *cluster_rest = on ? bt->cluster2 : 0;
  if (threads_rest) *threads_rest = on ? bt->threads2 : 0;
  if (clusters_rest) *clusters_rest = on ? bt->clusters2 : 0;
  return PRCG_OK;
}

const char* prcg_batched_last_error(const prcg_batch* bt) { return bt ? bt->err.c_str() : ""; }

int prcg_batched_destroy(prcg_batch* bt) {
  if (!bt) return PRCG_OK;
  if (bt->cs) cudaStreamSynchronize(bt->cs);
  drop_graph(bt);
  cudaFree(bt->d_sys);
  cudaFree(bt->d_order);
  cudaFree(bt->d_iters);
  cudaFree(bt->d_status);
  cudaFree(bt->d_queue);
  cudaFree(bt->d_true);
  cudaFree(bt->pool);
  if (bt->ev_user) cudaEventDestroy(bt->ev_user);
  if (bt->ev0) cudaEventDestroy(bt->ev0);
  if (bt->ev1) cudaEventDestroy(bt->ev1);
  if (bt->ev_fork) cudaEventDestroy(bt->ev_fork);
  if (bt->ev_join) cudaEventDestroy(bt->ev_join);
  if (bt->cs2) cudaStreamDestroy(bt->cs2);
  if (bt->cs) cudaStreamDestroy(bt->cs);
  delete bt;
  return PRCG_OK;
}

}  // extern "C"
