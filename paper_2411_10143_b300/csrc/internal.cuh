// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <functional>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cascade.h"

namespace cp {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
// Timestamped trace line on stderr when the environment sets CASCADE_TRACE=1
// (prediction / conversion / solve-loop steps; off by default).
void trace(const char* fmt, ...);
bool trace_on();

struct Error {
  cp_status status;
};

#define CP_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      ::cp::set_error("%s failed at %s:%d: %s", #call, __FILE__, __LINE__,            \
                      cudaGetErrorString(e_));                                        \
      throw ::cp::Error{e_ == cudaErrorMemoryAllocation ? CP_ERR_OOM : CP_ERR_CUDA};  \
    }                                                                                 \
  } while (0)

#define CP_REQUIRE(cond, st, ...)   \
  do {                              \
    if (!(cond)) {                  \
      ::cp::set_error(__VA_ARGS__); \
      throw ::cp::Error{st};        \
    }                               \
  } while (0)

// Every kernel launch goes through this, so the context counts launches and a
// bad launch configuration is reported at once.
#define CP_LAUNCH(ctx, kernel, grid, block, smem, stream, ...)  \
  do {                                                          \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);  \
    (ctx)->launches.fetch_add(1, std::memory_order_relaxed);    \
    CP_CUDA(cudaGetLastError());                                \
  } while (0)

// ---------------------------------------------------------------- device memory
template <typename T>
T* dalloc(size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  CP_CUDA(cudaMalloc(&p, count * sizeof(T)));
  return static_cast<T*>(p);
}
inline void dfree(void* p) {
  if (p) cudaFree(p);
}

// Stream-ordered temporaries: unlike cudaFree, cudaFreeAsync does not wait for
// the whole device, so conversions on the side stream never stall behind the
// solve running on the main stream.
template <typename T>
T* dalloc_async(size_t count, cudaStream_t s) {
  void* p = nullptr;
  if (count == 0) count = 1;
  CP_CUDA(cudaMallocAsync(&p, count * sizeof(T), s));
  return static_cast<T*>(p);
}
inline void dfree_async(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

constexpr int kBlock = 256;         // threads per block of the streaming kernels
constexpr int kMaxPartials = 4096;  // capacity of one block-partials buffer
constexpr int kMergeItems = 7;      // merge-path items per thread
constexpr int kMergeTile = kBlock * kMergeItems;  // block tile (allocation-free kernel)
constexpr int kMergeWarpTile = 32 * kMergeItems;  // warp tile (the matrix path's kernel)

struct ModelSlot {
  bool loaded = false;
  int h1 = 0, h2 = 0, k = 0;
  uint64_t gen = 0;           // installation number, unique in the process
  float* d_params = nullptr;  // device, flat layout of cascade.h
  float* d_mu = nullptr;      // device [15]
  float* d_sd = nullptr;      // device [15]
};

struct EllPart {
  int64_t K = 0, ld = 0;
  int32_t* col = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
};
struct CooPart {
  int64_t n = 0;
  int32_t* row = nullptr;
  int32_t* col = nullptr;  // aliases the CSR array for plain COO (owns_colval false)
  double* val = nullptr;
  float* val32 = nullptr;
  bool owns_colval = false;
};
struct SellPart {
  int64_t C = 0, sigma = 0, nchunks = 0, slots = 0;
  int32_t* perm = nullptr;
  int32_t* chunk_len = nullptr;
  int64_t* chunk_ptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
};

struct DiaPart {
  int64_t ndiag = 0;
  int32_t* offs = nullptr;  // ascending col - row
  double* val = nullptr;    // [ndiag][nrows]
  float* val32 = nullptr;
};
constexpr int kDiaMax = 1024;  // most diagonals a DIA conversion accepts

}  // namespace cp

namespace cp {
// The side thread of the asynchronous mode ("thread 2" of Sec. III-C-2), kept
// alive for the context's lifetime and bound to its GPU, so that starting the
// Host-mapped pages a context reuses across solves (each solve's mirror and
// yield flag).  cudaHostAlloc takes hundreds of microseconds and cudaFreeHost
// waits for the device, both inside a solve's time, so the pages are kept.
class MappedPool {
 public:
  static constexpr size_t kPage = 4096;
  void* take() {  // a zeroed page; its device view is cudaHostGetDevicePointer's
    void* p = nullptr;
    {
      std::lock_guard<std::mutex> lock(mu_);
      if (!free_.empty()) {
        p = free_.back();
        free_.pop_back();
      }
    }
    if (!p) {
      CP_CUDA(cudaHostAlloc(&p, kPage, cudaHostAllocMapped));
      std::lock_guard<std::mutex> lock(mu_);
      all_.push_back(p);
    }
    std::memset(p, 0, kPage);
    return p;
  }
  void give(void* p) {
    std::lock_guard<std::mutex> lock(mu_);
    free_.push_back(p);
  }
  void release() {  // at context destruction, with no solve running
    for (void* p : all_) cudaFreeHost(p);
    all_.clear();
    free_.clear();
  }

 private:
  std::mutex mu_;
  std::vector<void*> free_, all_;
};

// CUDA events a context reuses across solves (the profiling pairs around SpMV
// launches, the host's look-ahead ring, the persistent launches' timers).
class EventPool {
 public:
  cudaEvent_t take(bool timing) {
    {
      std::lock_guard<std::mutex> lock(mu_);
      auto& v = timing ? timing_ : plain_;
      if (!v.empty()) {
        cudaEvent_t e = v.back();
        v.pop_back();
        return e;
      }
    }
    cudaEvent_t e = nullptr;
    CP_CUDA(cudaEventCreateWithFlags(&e, timing ? cudaEventDefault : cudaEventDisableTiming));
    return e;
  }
  void give(cudaEvent_t e, bool timing) {
    std::lock_guard<std::mutex> lock(mu_);
    (timing ? timing_ : plain_).push_back(e);
  }
  void release() {
    for (auto e : timing_) cudaEventDestroy(e);
    for (auto e : plain_) cudaEventDestroy(e);
    timing_.clear();
    plain_.clear();
  }

 private:
  std::mutex mu_;
  std::vector<cudaEvent_t> timing_, plain_;
};

// cascade costs a wake-up (tens of microseconds), not a thread creation and a
// device binding (up to a millisecond, longer than a small solve).  One job at
// a time: post() hands it over, wait() returns when it has finished.
class SideWorker {
 public:
  explicit SideWorker(int device);
  ~SideWorker();
  void post(std::function<void()> job);
  void wait();

 private:
  void loop(int device);
  std::mutex mu_;
  std::condition_variable cv_;
  std::function<void()> job_;
  bool busy_ = false, stop_ = false;
  std::thread th_;
};
}  // namespace cp

namespace cp {
struct BatchGraphs;
// Releases the context's batched-solve graphs (cp_destroy).
void batch_graphs_release(cp_ctx* ctx);
}  // namespace cp

struct cp_ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t main = nullptr, side = nullptr;
  bool own_main = false, own_side = false;
  std::atomic<int64_t> launches{0};
  int64_t format_budget = int64_t(4) << 30;
  int grid_stream = 0;  // resident blocks of kBlock threads for streaming kernels
  cp::ModelSlot models[CP_NUM_STAGES];
  std::mutex model_mu;
  // pinned staging for small device-to-host reads, one per stream: a copy into
  // pageable memory can serialise behind the legacy default stream, which
  // would stall the side stream's prediction behind a running solve
  void* pin_main = nullptr;
  void* pin_side = nullptr;
  cp_gate gate{};  // cost-aware switching (disabled until installed)
  // per-matrix speedups for the gate (cp_gate_set_neighbours): the training
  // matrices' standardised features and per-format speedups
  struct GateNeighbours {
    int count = 0, k = 0;
    double mu[15] = {0}, sd[15] = {0};
    std::vector<float> z, speedup;
  } gate_nb;
  std::mutex gate_mu;  // guards gate_nb (installed by the caller, read by the side thread)
  std::atomic<int> inject_side_fail{-1};  // host fault injection point (tests), -1: none
  cp::SideWorker* side_worker = nullptr;
  cp::MappedPool mapped;  // host-mapped pages reused by the solves
  cp::EventPool events;   // CUDA events reused by the solves
  cp::BatchGraphs* batch_graphs = nullptr;  // instantiated batched-solve graphs (batch.cu)
  // a serving lane's context: the server's count of lanes holding a job.  Its
  // solves use the persistent (cooperative) kernels only while it is the one
  // busy lane, and ask a running one to return when another lane gets work, so
  // no two cooperative grids ever share the device (null: not a serving lane)
  const std::atomic<int>* lanes_busy = nullptr;
};

struct cp_mat {
  cp_ctx* ctx = nullptr;
  int64_t nrows = 0, ncols = 0, nnz = 0;
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;  // FP32 copy of val, made on first FP32 use
  bool has_coo = false, has_ell = false, has_sell = false, has_hyb = false, has_dia = false;
  cp::CooPart coo;
  cp::EllPart ell;
  cp::SellPart sell;
  cp::EllPart hyb_ell;
  cp::CooPart hyb_coo;
  int64_t hyb_auto_k = 0;  // HYB's width for hyb_k = 0, found on first use
  cp::DiaPart dia;
  bool has_features = false;
  double features[15] = {0};
  // the batched solve's threads per row for this matrix, from the BATCH_TPR
  // classifier installation numbered batch_tpr_gen (0: none yet); under feat_mu
  int batch_tpr = 0;
  uint64_t batch_tpr_gen = 0;
  // the diagonal offsets present (bit col - row + nrows - 1), left by the
  // feature pass for the DIA conversion; published once complete
  std::atomic<unsigned*> diag_bm{nullptr};
  // merge-path scratch: one carry (row, value) per tile
  int32_t* merge_carry_row = nullptr;
  double* merge_carry_val = nullptr;
  int32_t* merge_start = nullptr;  // row index where each tile's merge path starts (tiles + 1)
  int64_t merge_tiles = 0;
  // a host-mapped word the merge-path kernel sets when a bounded wait for its
  // tile copies gives up (host view, device view; from the context's page pool)
  int* merge_err = nullptr;
  int* merge_err_dev = nullptr;
  std::mutex mu;       // serialises conversions issued by the side thread and the caller
  std::mutex feat_mu;  // serialises the feature computation
};

namespace cp {

// ---------------------------------------------------------------- library-internal API
void csr_validate(cp_ctx* ctx, cp_mat* m);
void compute_features(cp_ctx* ctx, cp_mat* m, cudaStream_t s, double* out15);
void ensure_format(cp_ctx* ctx, cp_mat* m, const cp_config& cfg, cudaStream_t s);
void ensure_val32(cp_ctx* ctx, cp_mat* m, const cp_config& cfg, cudaStream_t s);
void format_dims(cp_mat* m, const cp_config& cfg, int64_t dims[4]);
void format_export(cp_mat* m, const cp_config& cfg, int array_id, void* dst, int64_t cap,
                   int64_t* bytes, cudaStream_t s);
void free_formats(cp_mat* m);
void config_check(const cp_config& c);  // throws CP_ERR_UNSUPPORTED
bool config_equal(const cp_config& a, const cp_config& b);
int64_t hyb_width(cp_ctx* ctx, cp_mat* m, const cp_config& c, cudaStream_t s);

// SpMV for the solvers: y = A x and, when dotv is non-null, block partial sums
// of y .* dotv written to partials[0..P); returns P (0 without dotv).
// The format of cfg must have been converted (and, for T = float, its FP32
// values made).  T is double or float.
// skip: device flag (may be null); when it is set the kernels return at once.
template <typename T>
int spmv_solver(cp_ctx* ctx, cp_mat* m, const cp_config& cfg, const T* x, T* y, const T* dotv,
                double* partials, const int* skip, cudaStream_t s);
// Block partial sums of a .* b (one per block of the resident grid); returns P.
template <typename T>
int dot_partials(cp_ctx* ctx, int64_t n, const T* a, const T* b, double* partials,
                 const int* skip, cudaStream_t s);
// General y = alpha A x + beta y.
// merge_start[t] for every tile boundary t = 0..tiles (one search per boundary)
void merge_partition(cp_ctx* ctx, cp_mat* m, cudaStream_t s);
// shared-memory carve-out of the kernels that stage tiles in shared memory
void spmv_set_attributes();

template <typename T>
void spmv_general(cp_ctx* ctx, cp_mat* m, const cp_config& cfg, T alpha, const T* x, T beta,
                  T* y, cudaStream_t s);

// Copy `bytes` (<= 4096) of device memory to host `dst` through the stream's
// pinned staging buffer and wait for the stream.
void d2h_small(cp_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t s);

// Exclusive scan of int64 counts in[0..n) into out[0..n] (out[n] = total).
void exclusive_scan_i64(cp_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);

}  // namespace cp

#include <vector>

namespace cp {

// Hand-off from the prediction side (feature extraction, cascade stages and
// conversions on the side stream, driven by a host thread) to the solve loop.
// A configuration is published only after the conversion it needs has
// completed on the side stream, so the solve loop may use it at once.
struct Mirror;  // persist.cuh

struct Channel {
  std::mutex mu;
  std::vector<std::pair<int, cp_config>> published;  // (stage, configuration) in order
  std::atomic<int> count{0};
  std::atomic<bool> cancel{false};
  std::atomic<bool> finished{false};  // the side work has ended (all stages, cancel or error)
  // the side thread is only waiting on the host (the cost-aware gate's
  // windows): the solve may run its persistent kernel meanwhile, and asks it
  // to return as soon as this goes false (the side stream needs the GPU)
  std::atomic<bool> side_gpu_idle{false};
  bool need_fp32 = false;  // the solve also needs FP32 values of every published format
  float t_features_ms = 0.f, t_predict_ms[3] = {0.f, 0.f, 0.f}, t_convert_ms = 0.f;
  cp_status status = CP_OK;  // first error of the side thread, if any
  std::string error;
  // the solve's progress for the cost-aware gate (FP64 solves): the solve's
  // host-mapped mirror, which the GPU updates as iterations complete (null
  // until the solve has set it up)
  std::atomic<const Mirror*> live{nullptr};
  std::atomic<bool> solve_done{false};
  double tol = 0.0;
  int gate_declined = 0;  // 1: kept the default after FORMAT; 2: skipped the feature pass
  float gate_remaining = -1.f, gate_cost = -1.f;

  void publish(int stage, const cp_config& c) {
    std::lock_guard<std::mutex> lock(mu);
    published.emplace_back(stage, c);
    count.store((int)published.size(), std::memory_order_release);
  }
};

// The cascaded prediction of Sec. III-C-1 (Fig. 5) with its conversions, on
// stream s; publishes into ch after every stage that changes the
// configuration.  Runs until done or ch->cancel is set.
void run_cascade(cp_ctx* ctx, cp_mat* m, cudaStream_t s, Channel* ch);
// the median speedup of format fmt over the k training matrices nearest to
// features (cp_gate_knn_speedup); arguments already checked
double gate_knn_speedup(int count, int k, const double* mu, const double* sd, const float* z,
                        const float* speedup, const double* features, int fmt);
// the cost-aware gate's rule (see cp_gate_decide)
int gate_decide(const cp_gate& g, int fmt, int64_t nnz, int iters, double res0, double res,
                double target, double* remaining, double* cost);
// default-kernel iterations after which switching to fmt has paid for its
// conversion (see cp_gate_payback)
double gate_payback(const cp_gate& g, int fmt, int64_t nnz);
// One cascade stage's classifier on the features: returns the arg-max class,
// or -1 when the stage has no model.
// One cascade stage's classifier (k_mlp_infer) on a feature vector: returns the
// arg-max class (-1 without a model); logits (host, k floats, may be NULL)
// receives the stage's logits.
int infer_stage(cp_ctx* ctx, int stage, const double* f15, cudaStream_t s,
                float* logits = nullptr);
// Classes of the stage's installed model (0 if none).
int stage_classes(cp_ctx* ctx, int stage);

// ---------------------------------------------------------------- predictor MLP
struct MlpDims {
  int d, h1, h2, k;
  __host__ __device__ int64_t nparams() const {
    return (int64_t)h1 * d + h1 + (int64_t)h2 * h1 + h2 + (int64_t)k * h2 + k;
  }
};
void mlp_forward(cp_ctx* ctx, int64_t N, MlpDims D, const float* P, const float* X, float* Z,
                 float* scratch, cudaStream_t s);
// targets: class labels lab[N], or target distributions Q[N][k] (one of the two)
void mlp_loss_grad(cp_ctx* ctx, int64_t N, MlpDims D, const float* P, const float* X,
                   const int32_t* lab, const float* Q, float* loss, float* grad, float* scratch,
                   cudaStream_t s);
void adam_step(cp_ctx* ctx, int64_t np, float* P, const float* G, float* m, float* v, int t,
               float lr, float b1, float b2, float eps, cudaStream_t s);
// gen: the installation number to record (0: a new one; a copy of another
// context's model passes that model's, so picks kept with a matrix stay valid)
void model_install(cp_ctx* ctx, int stage, int h1, int h2, int k, const float* params,
                   const float* mu, const float* sd, cudaStream_t s, uint64_t gen = 0);
void model_train(cp_ctx* ctx, int stage, int64_t N, const double* F_host,
                 const int32_t* lab_host, const float* q_host, int h1, int h2, int k, int epochs,
                 float lr, uint64_t seed, float* final_loss);
int64_t scratch_floats_api(int64_t N, int d, int h1, int h2, int k);

// A batched launch's shape: threads per system and threads per row.
struct BatchSchedule {
  int threads;
  int tpv;
  int order = 0;  // packing: 0 = largest systems first, 1 = in the caller's order
};
// threads / tpv = 0: the schedule of the batch's class (tuned, else by size)
void batch_solve(cp_ctx* ctx, int nsys, cp_mat* const* mats, const int32_t* solver,
                 const double* const* b, double* const* x, const cp_solve_opts* o,
                 cp_solve_info* infos, int threads, int tpv);
// the autotuner: times 128/256/512/1024 threads per system x 1/4/16 threads per
// row on this batch (scratch solutions, largest systems first), then the best
// shape in the caller's order; records the fastest for the batch's class,
// returns it; ms12[threads index * 3 + tpv index], ms_order (may be null) the
// best shape in the caller's order
BatchSchedule batch_tune(cp_ctx* ctx, int nsys, cp_mat* const* mats, const int32_t* solver,
                         const double* const* b, const cp_solve_opts* o, float* ms12,
                         float* ms_order);
// the schedule cp_batch_solve uses for a batch class (tuned, else by size)
BatchSchedule batch_schedule(cp_ctx* ctx, int64_t mean_rows, bool has_gmres);
// the BATCH_TPR classifier's threads per row for m (cp_batch_tpr), 0 without a model
int batch_tpr_of(cp_ctx* ctx, cp_mat* m, cudaStream_t s);
// a number that changes whenever a model is installed for `stage` in ctx (0:
// the stage has no model)
uint64_t model_generation(cp_ctx* ctx, int stage);

// The solve entry (CG or GMRES; FP64 or FP32-inner refinement; plain,
// sequential or asynchronous prediction).
void solve(cp_ctx* ctx, cp_mat* m, const double* b, double* x, const cp_solve_opts* o,
           cp_solve_info* info, bool gmres);

}  // namespace cp
