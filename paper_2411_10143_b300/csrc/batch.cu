// Batched persistent solves: many small systems in one launch.
//
// One thread block solves one system at a time and takes the next from a
// device work counter until the batch is empty (a persistent launch: the grid
// is sized to the resident capacity, not to the batch).  Each system runs FP64
// iterative refinement around FP32 inner solves, CG or GMRES(m) per system:
// the FP64 residual r = b - A x, the refinement update and GMRES's Givens /
// least-squares step in FP64, the SpMV and Krylov vectors in FP32.  Every
// reduction is a block reduction; no host round trip happens inside a solve.
// The single persistent launch is captured in a CUDA graph and launched as one.
// Threads per system come from a per-device schedule that cp_batch_tune fills
// by timing the candidates on real batches (the autotuner), else from the
// mean system size.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace cp {

constexpr int kBatchMaxM = 32;  // GMRES restart length limit inside a block

struct BatchSys {
  int64_t n;
  const int32_t* rowptr;
  const int32_t* col;
  const double* val;
  const float* val32;
  const double* b;
  double* x;
  double* r;     // [n] FP64 residual
  float* w32;    // FP32 workspace: CG 4n (r, d, p, ap); GMRES (m + 2) n (V, d)
  int solver;    // 0 CG, 1 GMRES
  int tpr;       // threads per row of this system's row loops: 1, 4 or 16
};

struct BatchOut {
  int status;
  int outer;
  int inner;
  double relres;
};

struct BatchParams {
  double tol, inner_tol;
  int max_outer, max_inner, m;
  double theta;  // an inner solve also stops at residual theta tol ||b||
};

// ------------------------------------------------------------------ block helpers
template <int BT>
__device__ __forceinline__ double bsum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < BT / 32 ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Block sum; thread 0 also forms g(total) (a quotient: FP64 divisions are
// instruction sequences on the FP64 pipe, so one thread forms them); both go
// to every thread.
template <int BT, typename G>
__device__ __forceinline__ double2 bsum_g(double v, double* red, G g) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < BT / 32 ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) {
      red[32] = s;
      red[33] = g(s);
    }
  }
  __syncthreads();
  return make_double2(red[32], red[33]);
}

// Row loops of the batched kernel: TPV threads per row (1: a thread per row,
// CSR-scalar; 4 or 16: groups of lanes share a row's entries and add their
// partial sums with shuffles, for systems with long rows).  The loop over row
// blocks runs the same number of trips in every thread, so whole warps reach
// the shuffles.
template <int BT, int TPV, typename F>
__device__ __forceinline__ void for_rows(int64_t n, F&& f) {
  if constexpr (TPV == 1) {
    for (int64_t i = threadIdx.x; i < n; i += BT) f(i, 0, true);
  } else {
    constexpr int RPB = BT / TPV;
    const int sub = threadIdx.x % TPV;
    for (int64_t base = 0; base < n; base += RPB) {
      const int64_t i = base + threadIdx.x / TPV;
      f(i, sub, i < n);
    }
  }
}
template <int TPV, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = TPV / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP64 residual r = b - A x (FP64 values) and ||r||^2
template <int BT, int TPV>
__device__ double resid64(const BatchSys& S, double* red) {
  double acc = 0.0;
  for_rows<BT, TPV>(S.n, [&](int64_t i, int sub, bool in) {
    double s = 0.0;
    if (in)
      for (int k = S.rowptr[i] + sub; k < S.rowptr[i + 1]; k += TPV)
        s = fma(S.val[k], S.x[S.col[k]], s);
    s = group_sum<TPV>(s);
    if (in && sub == 0) {
      const double ri = S.b[i] - s;
      S.r[i] = ri;
      acc = fma(ri, ri, acc);
    }
  });
  return bsum<BT>(acc, red);
}

// y = A32 v (FP32)
template <int BT, int TPV>
__device__ __forceinline__ void spmv32(const BatchSys& S, const float* v, float* y) {
  for_rows<BT, TPV>(S.n, [&](int64_t i, int sub, bool in) {
    float s = 0.f;
    if (in)
      for (int k = S.rowptr[i] + sub; k < S.rowptr[i + 1]; k += TPV)
        s = fmaf(S.val32[k], v[S.col[k]], s);
    s = group_sum<TPV>(s);
    if (in && sub == 0) y[i] = s;
  });
}

// ------------------------------------------------------------------ inner CG (FP32)
template <int BT, int TPV>
__device__ int inner_cg(const BatchSys& S, const BatchParams& P, int budget, double* red,
                        double floor2 /* (theta tol ||b||)^2 */) {
  const int64_t n = S.n;
  float* r = S.w32;
  float* d = r + n;
  float* p = d + n;
  float* ap = p + n;
  double rr = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += BT) {
    const float ri = __double2float_rn(S.r[i]);
    r[i] = ri;
    p[i] = ri;
    d[i] = 0.f;
    rr = fma((double)ri, (double)ri, rr);
  }
  rr = bsum<BT>(rr, red);
  const double stop = fmax(P.inner_tol * P.inner_tol * rr, floor2);
  int it = 0;
  // Each thread accumulates its share of a dot product in FP32 (a few dozen
  // terms at most: the inner solve is FP32 throughout); the block adds the
  // shares in FP64.
  while (it < budget && rr > stop) {
    __syncthreads();
    spmv32<BT, TPV>(S, p, ap);
    __syncthreads();
    float pap_t = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += BT) pap_t = fmaf(p[i], ap[i], pap_t);
    // alpha = rr / (p, Ap); -1 flags a breakdown (A not SPD)
    const double alpha_d =
        bsum_g<BT>((double)pap_t, red, [rr](double pap) { return pap > 0.0 ? rr / pap : -1.0; }).y;
    if (alpha_d < 0.0) return -1 - it;
    const float alpha = (float)alpha_d;
    float rn_t = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += BT) {
      d[i] = fmaf(alpha, p[i], d[i]);
      const float ri = fmaf(-alpha, ap[i], r[i]);
      r[i] = ri;
      rn_t = fmaf(ri, ri, rn_t);
    }
    const double2 rb = bsum_g<BT>((double)rn_t, red, [rr](double rn) { return rn / rr; });
    const float beta = (float)rb.y;
    rr = rb.x;
    for (int64_t i = threadIdx.x; i < n; i += BT) p[i] = fmaf(beta, p[i], r[i]);
    ++it;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += BT) S.x[i] += (double)d[i];
  return it;
}

// ------------------------------------------------------------------ inner GMRES (FP32 basis)
template <int BT, int TPV>
__device__ int inner_gmres(const BatchSys& S, const BatchParams& P, int budget, double* red,
                           double* Hs /*(m+1)*m*/, double* gs /*m+1*/, double* cs, double* sn,
                           double* hv /*m+1*/, float* acc_red /*32*(BT/32)*/,
                           double floor2 /* (theta tol ||b||)^2 */) {
  const int64_t n = S.n;
  const int m = P.m;
  float* V = S.w32;               // (m+1) columns of n
  float* d = V + (int64_t)(m + 1) * n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // inner rhs r32 = (float) r, x0 = 0: V0 = r32 / ||r32||
  double bb = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += BT) {
    const float ri = __double2float_rn(S.r[i]);
    V[i] = ri;
    d[i] = 0.f;
    bb = fma((double)ri, (double)ri, bb);
  }
  bb = bsum<BT>(bb, red);
  const double stop = fmax(P.inner_tol * sqrt(bb), sqrt(floor2));
  int it = 0;
  double beta = sqrt(bb);
  bool first = true;
  while (it < budget) {
    if (!first) {  // restart: V0 = r32 - A d
      __syncthreads();
      spmv32<BT, TPV>(S, d, V + n);  // scratch column 1
      __syncthreads();
      double s = 0.0;
      for (int64_t i = threadIdx.x; i < n; i += BT) {
        const float v0 = __double2float_rn(S.r[i]) - V[n + i];
        V[i] = v0;
        s = fma((double)v0, (double)v0, s);
      }
      beta = sqrt(bsum<BT>(s, red));
    }
    first = false;
    if (beta <= stop || beta == 0.0) break;
    const float inv = (float)(1.0 / beta);
    for (int64_t i = threadIdx.x; i < n; i += BT) V[i] *= inv;
    if (threadIdx.x == 0) {
      for (int q = 0; q <= m; ++q) gs[q] = 0.0;
      gs[0] = beta;
    }
    int jd = 0;
    bool conv = false;
    for (int j = 0; j < m && it < budget; ++j) {
      float* w = V + (int64_t)(j + 1) * n;
      __syncthreads();
      spmv32<BT, TPV>(S, V + (int64_t)j * n, w);
      if (threadIdx.x <= j) hv[threadIdx.x] = 0.0;
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        __syncthreads();
        float a[kBatchMaxM];
#pragma unroll
        for (int c = 0; c < kBatchMaxM; ++c) a[c] = 0.f;
        for (int64_t i = threadIdx.x; i < n; i += BT) {
          const float wi = w[i];
#pragma unroll
          for (int c = 0; c < kBatchMaxM; ++c)
            if (c <= j) a[c] = fmaf(V[(int64_t)c * n + i], wi, a[c]);
        }
#pragma unroll
        for (int c = 0; c < kBatchMaxM; ++c) a[c] = warp_sum(a[c]);
        if (lane == 0)
#pragma unroll
          for (int c = 0; c < kBatchMaxM; ++c) acc_red[c * (BT / 32) + warp] = a[c];
        __syncthreads();
        if (threadIdx.x <= j) {
          double s = 0.0;
          for (int q = 0; q < BT / 32; ++q) s += (double)acc_red[threadIdx.x * (BT / 32) + q];
          red[64 + threadIdx.x] = s;  // this pass's coefficient
          hv[threadIdx.x] += s;
        }
        __syncthreads();
        float wn_t = 0.f;
        for (int64_t i = threadIdx.x; i < n; i += BT) {
          float wi = w[i];
          for (int c = 0; c <= j; ++c) wi = fmaf(-(float)red[64 + c], V[(int64_t)c * n + i], wi);
          w[i] = wi;
          wn_t = fmaf(wi, wi, wn_t);
        }
        const double wn = bsum<BT>((double)wn_t, red);
        if (pass == 1 && threadIdx.x == 0) red[40] = wn;
      }
      // Givens rotation in FP64 (thread 0)
      if (threadIdx.x == 0) {
        const double hn = sqrt(red[40]);
        for (int i = 0; i <= j; ++i) Hs[i * m + j] = hv[i];
        for (int i = 0; i < j; ++i) {
          const double a0 = Hs[i * m + j], b0 = Hs[(i + 1) * m + j];
          Hs[i * m + j] = cs[i] * a0 + sn[i] * b0;
          Hs[(i + 1) * m + j] = -sn[i] * a0 + cs[i] * b0;
        }
        const double a0 = Hs[j * m + j];
        const double den = sqrt(a0 * a0 + hn * hn);
        cs[j] = den == 0.0 ? 1.0 : a0 / den;
        sn[j] = den == 0.0 ? 0.0 : hn / den;
        Hs[j * m + j] = cs[j] * a0 + sn[j] * hn;
        gs[j + 1] = -sn[j] * gs[j];
        gs[j] = cs[j] * gs[j];
        red[41] = hn;
        red[42] = fabs(gs[j + 1]);
        red[43] = hn > 0.0 ? 1.0 / hn : 0.0;
      }
      __syncthreads();
      const double hn = red[41];
      ++it;
      jd = j + 1;
      if (red[42] <= stop || hn == 0.0) {
        conv = red[42] <= stop;
        break;
      }
      const float inv2 = (float)red[43];
      for (int64_t i = threadIdx.x; i < n; i += BT) w[i] *= inv2;
    }
    // y = R^{-1} g, d += V y
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = jd - 1; i >= 0; --i) {
        double s = gs[i];
        for (int k = i + 1; k < jd; ++k) s -= Hs[i * m + k] * hv[k];
        hv[i] = s / Hs[i * m + i];  // hv reused as y
      }
    }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += BT) {
      float di = d[i];
      for (int c = 0; c < jd; ++c) di = fmaf((float)hv[c], V[(int64_t)c * n + i], di);
      d[i] = di;
    }
    if (conv) break;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += BT) S.x[i] += (double)d[i];
  return it;
}

// ------------------------------------------------------------------ the persistent kernel
// Shared-memory work areas of one block, handed to the per-system solve.
struct BatchSmem {
  double* red;
  double* Hs;
  double *gs, *cs, *sn, *hv;
  float* acc_red;
};

// One system, start to finish, with TPV threads per row.
template <int BT, int TPV>
__device__ void solve_system(const BatchSys& S, const BatchParams& P, const BatchSmem& W,
                             BatchOut* out, int id) {
  double* red = W.red;
  double bb = 0.0;
  for (int64_t i = threadIdx.x; i < S.n; i += BT) bb = fma(S.b[i], S.b[i], bb);
  bb = bsum<BT>(bb, red);
  int outer = 0, inner = 0, status = CP_OK;
  double rr = 0.0;
  for (;;) {
    __syncthreads();
    rr = resid64<BT, TPV>(S, red);
    if (bb == 0.0 || rr <= P.tol * P.tol * bb) break;
    if (!isfinite(rr)) {
      status = CP_ERR_BREAKDOWN;
      break;
    }
    if (outer >= P.max_outer || inner >= P.max_inner) {
      status = CP_ERR_NOT_CONVERGED;
      break;
    }
    __syncthreads();
    const int budget = P.max_inner - inner;
    const double floor2 = P.theta * P.theta * P.tol * P.tol * bb;
    int got = S.solver == 0 ? inner_cg<BT, TPV>(S, P, budget, red, floor2)
                            : inner_gmres<BT, TPV>(S, P, budget, red, W.Hs, W.gs, W.cs, W.sn,
                                                   W.hv, W.acc_red, floor2);
    if (got < 0) {
      status = CP_ERR_BREAKDOWN;
      inner += -got - 1;
      break;
    }
    inner += got;
    ++outer;
  }
  if (threadIdx.x == 0) {
    out[id].status = status;
    out[id].outer = outer;
    out[id].inner = inner;
    out[id].relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  }
}

// Every system carries its own threads per row (a block-uniform branch), so
// one launch can mix systems of short and of long rows.
template <int BT>
__global__ void __launch_bounds__(BT) k_batch_solve(const BatchSys* __restrict__ sys, int nsys,
                                                    const int* __restrict__ order,
                                                    int* __restrict__ next, BatchParams P,
                                                    BatchOut* __restrict__ out) {
  __shared__ double red[64 + kBatchMaxM + 1];
  __shared__ double Hs[(kBatchMaxM + 1) * kBatchMaxM];
  __shared__ double gs[kBatchMaxM + 1], cs[kBatchMaxM], sn[kBatchMaxM], hv[kBatchMaxM + 1];
  __shared__ float acc_red[kBatchMaxM * (BT / 32)];
  __shared__ int s_id;
  const BatchSmem W{red, Hs, gs, cs, sn, hv, acc_red};
  for (;;) {
    if (threadIdx.x == 0) s_id = atomicAdd(next, 1);
    __syncthreads();
    const int q = s_id;
    __syncthreads();
    if (q >= nsys) break;
    const int id = order[q];
    const BatchSys S = sys[id];
    if (S.tpr == 16) solve_system<BT, 16>(S, P, W, out, id);
    else if (S.tpr == 4) solve_system<BT, 4>(S, P, W, out, id);
    else solve_system<BT, 1>(S, P, W, out, id);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host
// The batched solve is one persistent launch in a CUDA graph.  Each context
// instantiates the graph of each (block size, threads per row) once, on first
// use; later batches only update the kernel node's grid and arguments in the
// instantiated graph (cudaGraphExecKernelNodeSetParams) and launch it, with no
// capture or instantiation on the path of a batch.
}  // namespace cp

namespace {
constexpr int kBatchThreads[4] = {128, 256, 512, 1024};
constexpr int kBatchTpv[3] = {1, 4, 16};
}  // namespace

struct cp::BatchGraphs {
  struct One {
    cudaGraph_t graph = nullptr;
    cudaGraphNode_t node = nullptr;
    cudaGraphExec_t exec = nullptr;
  };
  One by_bt[4];  // by threads per system
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace cp {

void batch_graphs_release(cp_ctx* ctx) {
  BatchGraphs* G = ctx->batch_graphs;
  if (!G) return;
  for (auto& o : G->by_bt) {
    if (o.exec) cudaGraphExecDestroy(o.exec);
    if (o.graph) cudaGraphDestroy(o.graph);
  }
  if (G->e0) cudaEventDestroy(G->e0);
  if (G->e1) cudaEventDestroy(G->e1);
  delete G;
  ctx->batch_graphs = nullptr;
}

static int bt_slot(int bt) { return bt == 128 ? 0 : bt == 256 ? 1 : bt == 512 ? 2 : 3; }

// Runs one batch with BT threads per system (each system's threads per row
// are in its descriptor); returns the launch's time (ms, CUDA events around
// the graph launch on s).
template <int BT>
static float launch_batch(cp_ctx* ctx, const BatchSys* d_sys, int nsys, const int* d_order,
                          int* d_next, const BatchParams& P, BatchOut* d_out, cudaStream_t s) {
  int per_sm = 0;
  CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_solve<BT>, BT, 0));
  int grid = ctx->num_sms * std::max(per_sm, 1);
  if (grid > nsys) grid = nsys;
  if (!ctx->batch_graphs) {
    BatchGraphs* G = new BatchGraphs;
    if (cudaEventCreate(&G->e0) != cudaSuccess || cudaEventCreate(&G->e1) != cudaSuccess) {
      ctx->batch_graphs = G;
      batch_graphs_release(ctx);
      CP_CUDA(cudaGetLastError());
      throw Error{CP_ERR_CUDA};
    }
    ctx->batch_graphs = G;
  }
  BatchGraphs::One& g = ctx->batch_graphs->by_bt[bt_slot(BT)];
  BatchSys const* a_sys = d_sys;
  int a_nsys = nsys;
  const int* a_order = d_order;
  int* a_next = d_next;
  BatchParams a_p = P;
  BatchOut* a_out = d_out;
  void* args[] = {&a_sys, &a_nsys, &a_order, &a_next, &a_p, &a_out};
  cudaKernelNodeParams kp{};
  kp.func = reinterpret_cast<void*>(k_batch_solve<BT>);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(BT);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  if (g.exec && cudaGraphExecKernelNodeSetParams(g.exec, g.node, &kp) != cudaSuccess) {
    // an update the instantiated graph does not take: build it again
    (void)cudaGetLastError();
    cudaGraphExecDestroy(g.exec);
    cudaGraphDestroy(g.graph);
    g = BatchGraphs::One{};
  }
  if (!g.exec) {
    CP_CUDA(cudaGraphCreate(&g.graph, 0));
    CP_CUDA(cudaGraphAddKernelNode(&g.node, g.graph, nullptr, 0, &kp));
    CP_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
  }
  ctx->launches.fetch_add(1, std::memory_order_relaxed);
  float ms = 0.f;
  CP_CUDA(cudaEventRecord(ctx->batch_graphs->e0, s));
  CP_CUDA(cudaGraphLaunch(g.exec, s));
  CP_CUDA(cudaEventRecord(ctx->batch_graphs->e1, s));
  CP_CUDA(cudaEventSynchronize(ctx->batch_graphs->e1));
  CP_CUDA(cudaEventElapsedTime(&ms, ctx->batch_graphs->e0, ctx->batch_graphs->e1));
  return ms;
}

static float launch_batch_cfg(int bt, cp_ctx* ctx, const BatchSys* d_sys, int nsys,
                              const int* d_order, int* d_next, const BatchParams& P,
                              BatchOut* d_out, cudaStream_t s) {
  switch (bt) {
    case 128: return launch_batch<128>(ctx, d_sys, nsys, d_order, d_next, P, d_out, s);
    case 256: return launch_batch<256>(ctx, d_sys, nsys, d_order, d_next, P, d_out, s);
    case 512: return launch_batch<512>(ctx, d_sys, nsys, d_order, d_next, P, d_out, s);
    default: return launch_batch<1024>(ctx, d_sys, nsys, d_order, d_next, P, d_out, s);
  }
}

// ---- the autotuner's schedule: (threads per system, threads per row) for a
// batch class, per device.  A class is (the batch holds a GMRES system,
// floor(log2(mean rows))).
namespace {
constexpr int kSchedDevices = 64;
constexpr int kSchedBuckets = 32;
std::mutex g_sched_mu;
BatchSchedule g_sched[kSchedDevices][2][kSchedBuckets] = {};  // threads 0: not tuned

int size_bucket(int64_t mean_rows) {
  int b = 0;
  while (b + 1 < kSchedBuckets && (int64_t(1) << (b + 1)) <= mean_rows) ++b;
  return b;
}

// Untuned rule.  The tuner measured 1024 threads fastest for batches of
// 32 mixed CG / GMRES systems of about 10,000 rows (52.8 ms against 94 / 175 /
// 341 ms with 512 / 256 / 128): a block per system leaves most SMs idle when
// the batch is smaller than the GPU, so wider blocks win early.  A thread per
// row (CSR-scalar).
BatchSchedule default_schedule(int64_t mean_rows) {
  return BatchSchedule{
      mean_rows < 512 ? 128 : mean_rows < 2048 ? 256 : mean_rows < 8192 ? 512 : 1024, 1};
}
}  // namespace

BatchSchedule batch_schedule(cp_ctx* ctx, int64_t mean_rows, bool has_gmres) {
  if (ctx->device >= 0 && ctx->device < kSchedDevices) {
    std::lock_guard<std::mutex> lock(g_sched_mu);
    const BatchSchedule t = g_sched[ctx->device][has_gmres ? 1 : 0][size_bucket(mean_rows)];
    if (t.threads) return t;
  }
  return default_schedule(mean_rows);
}

// A batch laid out on the device: per-system descriptors, workspaces, the
// largest-first work order and the outputs, all stream-ordered on s.
struct BatchJob {
  cudaStream_t s = nullptr;
  std::vector<BatchSys> hs;
  double* d64 = nullptr;
  float* d32 = nullptr;
  double* xs = nullptr;  // tuning: scratch solutions
  BatchSys* d_sys = nullptr;
  int* d_order = nullptr;  // nsys entries + the work counter
  BatchOut* d_out = nullptr;
  std::vector<int> order[2];  // largest systems first; the caller's order
  int64_t total_rows = 0;
  bool has_gmres = false;
  ~BatchJob() {
    dfree_async(d64, s);
    dfree_async(d32, s);
    dfree_async(xs, s);
    dfree_async(d_sys, s);
    dfree_async(d_order, s);
    dfree_async(d_out, s);
  }
};

static void batch_prepare(cp_ctx* ctx, BatchJob& J, int nsys, cp_mat* const* mats,
                          const int32_t* solver, const double* const* b, double* const* x,
                          const cp_solve_opts& opt, bool scratch_x) {
  CP_REQUIRE(nsys >= 1 && mats && solver && b && (x || scratch_x), CP_ERR_INVALID,
             "bad batch arguments");
  CP_REQUIRE(opt.restart >= 1 && opt.restart <= kBatchMaxM, CP_ERR_INVALID,
             "batched GMRES restart must be in 1..%d", kBatchMaxM);
  CP_REQUIRE(opt.ir_theta >= 0.0 && opt.ir_theta < 1.0, CP_ERR_INVALID,
             "ir_theta must be in [0, 1)");
  cudaStream_t s = J.s;
  cp_config csr;
  cp_config_default(&csr);
  int64_t ws64 = 0, ws32 = 0;
  for (int i = 0; i < nsys; ++i) {
    cp_mat* m = mats[i];
    CP_REQUIRE(m && m->nrows == m->ncols && b[i] && (scratch_x || x[i]), CP_ERR_INVALID,
               "system %d: NULL or non-square", i);
    CP_REQUIRE(solver[i] == 0 || solver[i] == 1, CP_ERR_INVALID, "system %d: solver must be 0/1",
               i);
    ensure_val32(ctx, m, csr, s);
    ws64 += m->nrows;
    ws32 += (solver[i] == 0 ? 4 : opt.restart + 2) * m->nrows;
    J.total_rows += m->nrows;
    J.has_gmres |= solver[i] == 1;
  }
  J.d64 = dalloc_async<double>(ws64, s);
  J.d32 = dalloc_async<float>(ws32, s);
  if (scratch_x) J.xs = dalloc_async<double>(J.total_rows, s);
  J.hs.resize(nsys);
  int64_t o64 = 0, o32 = 0;
  for (int i = 0; i < nsys; ++i) {
    cp_mat* m = mats[i];
    J.hs[i] = BatchSys{m->nrows, m->rowptr, m->col, m->val, m->val32, b[i],
                       scratch_x ? J.xs + o64 : x[i], J.d64 + o64, J.d32 + o32, solver[i], 1};
    o64 += m->nrows;
    o32 += (solver[i] == 0 ? 4 : opt.restart + 2) * m->nrows;
  }
  // packing orders of the dynamic queue: largest systems first (so the queue
  // ends with short jobs), or the caller's order
  J.order[1].resize(nsys);
  std::iota(J.order[1].begin(), J.order[1].end(), 0);
  J.order[0] = J.order[1];
  std::stable_sort(J.order[0].begin(), J.order[0].end(), [&](int a, int c) {
    return J.hs[a].n * (J.hs[a].solver ? 3 : 1) > J.hs[c].n * (J.hs[c].solver ? 3 : 1);
  });
  J.d_sys = dalloc_async<BatchSys>(nsys, s);
  J.d_order = dalloc_async<int>(nsys + 1, s);
  J.d_out = dalloc_async<BatchOut>(nsys, s);
  CP_CUDA(cudaStreamSynchronize(s));
}

// One launch of the batch with `threads` threads per system, tpr[i] threads
// per row for system i and packing order `order` (the descriptors and the
// order go to the device first; the launch synchronises, so J.hs may change
// before the next run).
static float batch_run(cp_ctx* ctx, BatchJob& J, int nsys, const cp_solve_opts& opt, int threads,
                       const std::vector<int>& tpr, int order) {
  cudaStream_t s = J.s;
  for (int i = 0; i < nsys; ++i) J.hs[i].tpr = tpr[i];
  CP_CUDA(cudaMemcpyAsync(J.d_sys, J.hs.data(), nsys * sizeof(BatchSys), cudaMemcpyHostToDevice,
                          s));
  CP_CUDA(cudaMemcpyAsync(J.d_order, J.order[order ? 1 : 0].data(), nsys * sizeof(int),
                          cudaMemcpyHostToDevice, s));
  if (J.xs) CP_CUDA(cudaMemsetAsync(J.xs, 0, J.total_rows * sizeof(double), s));
  CP_CUDA(cudaMemsetAsync(J.d_order + nsys, 0, sizeof(int), s));
  BatchParams P{opt.tol, opt.inner_tol, opt.max_outer, opt.maxit, opt.restart, opt.ir_theta};
  return launch_batch_cfg(threads, ctx, J.d_sys, nsys, J.d_order, J.d_order + nsys, P, J.d_out,
                          s);
}

// The CP_STAGE_BATCH_TPR classifier's threads per row for matrix m (1, 4 or
// 16), or 0 without a model.  The pick is kept with m, tagged with the model
// installation it came from.
int batch_tpr_of(cp_ctx* ctx, cp_mat* m, cudaStream_t s) {
  const uint64_t gen = model_generation(ctx, CP_STAGE_BATCH_TPR);
  if (!gen) return 0;
  {
    std::lock_guard<std::mutex> lock(m->feat_mu);
    if (m->batch_tpr_gen == gen) return m->batch_tpr;
  }
  double f[15];
  compute_features(ctx, m, s, f);
  const int k = infer_stage(ctx, CP_STAGE_BATCH_TPR, f, s);
  const int tpr = k == 2 ? 16 : k == 1 ? 4 : 1;
  std::lock_guard<std::mutex> lock(m->feat_mu);
  m->batch_tpr = tpr;
  m->batch_tpr_gen = gen;
  return tpr;
}

void batch_solve(cp_ctx* ctx, int nsys, cp_mat* const* mats, const int32_t* solver,
                 const double* const* b, double* const* x, const cp_solve_opts* o,
                 cp_solve_info* infos, int threads, int tpv) {
  cp_solve_opts opt;
  cp_solve_opts_default(&opt);
  if (o) opt = *o;
  CP_REQUIRE(threads == 0 || threads == 128 || threads == 256 || threads == 512 || threads == 1024,
             CP_ERR_INVALID, "threads per system must be 128, 256, 512 or 1024");
  CP_REQUIRE(tpv == 0 || tpv == 1 || tpv == 4 || tpv == 16, CP_ERR_INVALID,
             "threads per row must be 1, 4 or 16");
  BatchJob J;
  J.s = ctx->main;
  batch_prepare(ctx, J, nsys, mats, solver, b, x, opt, false);
  // threads = 0: the tuned (or default) schedule of the batch's class.  Threads
  // per row: tpv for every system when given, else each system's from the
  // BATCH_TPR classifier when it has a model, else the schedule's
  BatchSchedule sc = batch_schedule(ctx, J.total_rows / nsys, J.has_gmres);
  if (threads) sc = BatchSchedule{threads, 1, 0};
  std::vector<int> tpr(nsys, tpv ? tpv : sc.tpv);
  if (!tpv)
    for (int i = 0; i < nsys; ++i)
      if (const int t = batch_tpr_of(ctx, mats[i], J.s)) tpr[i] = t;
  const float launch_ms = batch_run(ctx, J, nsys, opt, sc.threads, tpr, sc.order);
  std::vector<BatchOut> out(nsys);
  CP_CUDA(cudaMemcpyAsync(out.data(), J.d_out, nsys * sizeof(BatchOut), cudaMemcpyDeviceToHost,
                          J.s));
  CP_CUDA(cudaStreamSynchronize(J.s));
  cp_config csr;
  cp_config_default(&csr);
  int worst = CP_OK;
  for (int i = 0; i < nsys; ++i) {
    if (infos) {
      std::memset(&infos[i], 0, sizeof(cp_solve_info));
      infos[i].iters = out[i].inner;
      infos[i].outer_iters = out[i].outer;
      infos[i].relres_true = out[i].relres;
      infos[i].status = out[i].status;
      infos[i].switch_iter[0] = infos[i].switch_iter[1] = infos[i].switch_iter[2] = -1;
      infos[i].final_cfg = csr;
      infos[i].t_total_ms = launch_ms;  // the whole batch's launch
    }
    if (out[i].status != CP_OK && worst == CP_OK) worst = out[i].status;
  }
  CP_REQUIRE(worst == CP_OK, (cp_status)worst, "a batched system did not converge (status %d)",
             worst);
}

BatchSchedule batch_tune(cp_ctx* ctx, int nsys, cp_mat* const* mats, const int32_t* solver,
                         const double* const* b, const cp_solve_opts* o, float* ms12,
                         float* ms_order) {
  cp_solve_opts opt;
  cp_solve_opts_default(&opt);
  if (o) opt = *o;
  BatchJob J;
  J.s = ctx->main;
  batch_prepare(ctx, J, nsys, mats, solver, b, nullptr, opt, true);
  BatchSchedule best{0, 1, 0};
  float best_ms = 0.f;
  for (int c = 0; c < 4; ++c)
    for (int v = 0; v < 3; ++v) {
      const BatchSchedule sc{kBatchThreads[c], kBatchTpv[v], 0};
      const std::vector<int> tpr(nsys, sc.tpv);
      batch_run(ctx, J, nsys, opt, sc.threads, tpr, 0);  // warm-up: module load, caches
      const float ms = batch_run(ctx, J, nsys, opt, sc.threads, tpr, 0);
      if (ms12) ms12[c * 3 + v] = ms;
      if (!best.threads || ms < best_ms) {
        best = sc;
        best_ms = ms;
      }
    }
  // the packing order at the best shape: the caller's order against largest first
  {
    const std::vector<int> tpr(nsys, best.tpv);
    batch_run(ctx, J, nsys, opt, best.threads, tpr, 1);
    const float ms = batch_run(ctx, J, nsys, opt, best.threads, tpr, 1);
    if (ms_order) *ms_order = ms;
    if (ms < best_ms) best.order = 1;
  }
  CP_CUDA(cudaStreamSynchronize(J.s));
  if (ctx->device >= 0 && ctx->device < kSchedDevices) {
    std::lock_guard<std::mutex> lock(g_sched_mu);
    g_sched[ctx->device][J.has_gmres ? 1 : 0][size_bucket(J.total_rows / nsys)] = best;
  }
  return best;
}

}  // namespace cp
