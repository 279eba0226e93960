// The C ABI of libcascade (declared in include/cascade.h): argument checks,
// error capture and dispatch into the runtime.  No entry point lets a C++
// exception or a CUDA error escape; each returns a cp_status and records a
// message for cp_last_error().
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <new>

#include "common.cuh"
#include "internal.cuh"

namespace cp {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

bool trace_on() {
  static const bool on = [] {
    const char* e = std::getenv("CASCADE_TRACE");
    return e && e[0] == '1';
  }();
  return on;
}

void trace(const char* fmt, ...) {
  if (!trace_on()) return;
  static const auto t0 = std::chrono::steady_clock::now();
  const double ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  std::fprintf(stderr, "[cascade %10.3f ms] %s\n", ms, buf);
}

template <typename F>
static cp_status guard(F&& f) {
  try {
    g_err[0] = 0;
    f();
    return CP_OK;
  } catch (const Error& e) {
    return e.status;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return CP_ERR_OOM;
  } catch (...) {
    set_error("unexpected internal error");
    return CP_ERR_CUDA;
  }
}

// Make ctx's device current for the calling thread.
static void use_device(cp_ctx* ctx) { CP_CUDA(cudaSetDevice(ctx->device)); }

}  // namespace cp

using namespace cp;

extern "C" {

void cp_config_default(cp_config* c) {
  if (!c) return;
  c->fmt = CP_FMT_CSR;
  c->algo = CP_ALGO_SCALAR;
  c->tpv = 8;
  c->sell_c = 32;
  c->sell_sigma = 1;
  c->hyb_k = 0;
}

void cp_solve_opts_default(cp_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->maxit = 100000;
  o->restart = 30;
  o->mode = CP_MODE_PLAIN;
  o->precision = CP_PREC_FP64;
  o->inner_tol = 1e-5;
  o->max_outer = 30;
  o->check_every = 8;
  o->profile = 0;
  o->force = nullptr;
  o->wait_limit_ms = 0.0;
  o->persist_chunk = 0;
  o->gmres_orth = 0;
  o->ir_theta = 0.5;
}

const char* cp_last_error(void) { return g_err; }

int64_t cp_abi_sizeof(int32_t which) {
  switch (which) {
    case 0: return (int64_t)sizeof(cp_config);
    case 1: return (int64_t)sizeof(cp_solve_opts);
    case 2: return (int64_t)sizeof(cp_solve_info);
    case 3: return (int64_t)sizeof(cp_gate);
    case 4: return (int64_t)sizeof(cp_server_opts);
    case 5: return (int64_t)sizeof(cp_request);
    case 6: return (int64_t)sizeof(cp_result);
    default: return -1;
  }
}

cp_status cp_create(cp_ctx** out, int32_t device, void* main_stream, void* side_stream) {
  return guard([&] {
    CP_REQUIRE(out, CP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int count = 0;
    CP_CUDA(cudaGetDeviceCount(&count));
    CP_REQUIRE(device >= 0 && device < count, CP_ERR_INVALID, "device %d not present (%d GPUs)",
               device, count);
    CP_CUDA(cudaSetDevice(device));
    cp_ctx* c = new cp_ctx();
    c->device = device;
    try {
      CP_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
      int max_threads = 0;
      CP_CUDA(cudaDeviceGetAttribute(&max_threads, cudaDevAttrMaxThreadsPerMultiProcessor, device));
      c->grid_stream = c->num_sms * (max_threads / kBlock);
      if (c->grid_stream > kMaxPartials) c->grid_stream = kMaxPartials;
      spmv_set_attributes();
      c->side_worker = new cp::SideWorker(device);
      if (main_stream) {
        c->main = static_cast<cudaStream_t>(main_stream);
      } else {
        CP_CUDA(cudaStreamCreateWithFlags(&c->main, cudaStreamNonBlocking));
        c->own_main = true;
      }
      if (side_stream) {
        c->side = static_cast<cudaStream_t>(side_stream);
      } else {
        CP_CUDA(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        c->own_side = true;
      }
      CP_CUDA(cudaHostAlloc(&c->pin_main, 4096, cudaHostAllocDefault));
      CP_CUDA(cudaHostAlloc(&c->pin_side, 4096, cudaHostAllocDefault));
      // keep memory freed by stream-ordered frees in this process's pool, so a
      // conversion on the side stream reuses it instead of growing the pool
      // (growth can wait for work already running on the device)
      cudaMemPool_t pool;
      CP_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
      uint64_t keep = UINT64_MAX;
      CP_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
      // the pool's first allocation is slow and can wait for running work: make it
      // here, before any solve, and keep 64 MiB reserved for side-stream temporaries
      void* warm = nullptr;
      CP_CUDA(cudaMallocAsync(&warm, size_t(64) << 20, c->side));
      CP_CUDA(cudaFreeAsync(warm, c->side));
      CP_CUDA(cudaStreamSynchronize(c->side));
    } catch (...) {
      delete c->side_worker;
      if (c->pin_main) cudaFreeHost(c->pin_main);
      if (c->pin_side) cudaFreeHost(c->pin_side);
      if (c->own_main && c->main) cudaStreamDestroy(c->main);
      if (c->own_side && c->side) cudaStreamDestroy(c->side);
      delete c;
      throw;
    }
    *out = c;
  });
}

namespace cp {
SideWorker::SideWorker(int device) : th_([this, device] { loop(device); }) {}

SideWorker::~SideWorker() {
  {
    std::lock_guard<std::mutex> lock(mu_);
    stop_ = true;
  }
  cv_.notify_all();
  th_.join();
}

void SideWorker::post(std::function<void()> job) {
  std::lock_guard<std::mutex> lock(mu_);
  job_ = std::move(job);
  busy_ = true;
  cv_.notify_all();
}

void SideWorker::wait() {
  std::unique_lock<std::mutex> lock(mu_);
  cv_.wait(lock, [this] { return !busy_; });
}

void SideWorker::loop(int device) {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lock(mu_);
  for (;;) {
    cv_.wait(lock, [this] { return stop_ || busy_; });
    if (busy_) {
      std::function<void()> job = std::move(job_);
      lock.unlock();
      job();  // run_cascade catches its own errors
      lock.lock();
      busy_ = false;
      cv_.notify_all();
    }
    if (stop_ && !busy_) return;
  }
}
}  // namespace cp

cp_status cp_destroy(cp_ctx* ctx) {
  return guard([&] {
    if (!ctx) return;
    use_device(ctx);
    delete ctx->side_worker;  // joins the side thread (idle between solves)
    ctx->side_worker = nullptr;
    cudaStreamSynchronize(ctx->main);
    cudaStreamSynchronize(ctx->side);
    for (auto& mslot : ctx->models) {
      dfree(mslot.d_params);
      dfree(mslot.d_mu);
      dfree(mslot.d_sd);
    }
    if (ctx->own_main) cudaStreamDestroy(ctx->main);
    if (ctx->own_side) cudaStreamDestroy(ctx->side);
    if (ctx->pin_main) cudaFreeHost(ctx->pin_main);
    if (ctx->pin_side) cudaFreeHost(ctx->pin_side);
    ctx->mapped.release();
    ctx->events.release();
    batch_graphs_release(ctx);
    delete ctx;
  });
}

cp_status cp_ctx_launch_count(cp_ctx* ctx, int64_t* count) {
  return guard([&] {
    CP_REQUIRE(ctx && count, CP_ERR_INVALID, "NULL argument");
    *count = ctx->launches.load();
  });
}

cp_status cp_set_format_budget(cp_ctx* ctx, int64_t bytes) {
  return guard([&] {
    CP_REQUIRE(ctx && bytes > 0, CP_ERR_INVALID, "bad budget");
    ctx->format_budget = bytes;
  });
}

cp_status cp_csr_load(cp_ctx* ctx, int64_t nrows, int64_t ncols, int64_t nnz,
                      const int32_t* rowptr, const int32_t* col, const double* val,
                      int32_t on_device, cp_mat** out) {
  return guard([&] {
    CP_REQUIRE(ctx && out && rowptr, CP_ERR_INVALID, "NULL argument");
    *out = nullptr;
    CP_REQUIRE(nrows >= 1 && ncols >= 1 && nrows < (int64_t(1) << 31) &&
                   ncols < (int64_t(1) << 31),
               CP_ERR_INVALID, "nrows and ncols must be in 1..2^31-1");
    CP_REQUIRE(nnz >= 0 && nnz < (int64_t(1) << 31), CP_ERR_INVALID, "nnz must be in 0..2^31-1");
    CP_REQUIRE(nnz == 0 || (col && val), CP_ERR_INVALID, "col/val are NULL");
    use_device(ctx);
    cp_mat* m = new cp_mat();
    m->ctx = ctx;
    m->nrows = nrows;
    m->ncols = ncols;
    m->nnz = nnz;
    try {
      // from the context's stream-ordered pool, which keeps its memory: a load
      // after the first spends no time mapping fresh device memory
      m->rowptr = dalloc_async<int32_t>(nrows + 1, ctx->main);
      m->col = dalloc_async<int32_t>(nnz, ctx->main);
      m->val = dalloc_async<double>(nnz, ctx->main);
      const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
      CP_CUDA(cudaMemcpyAsync(m->rowptr, rowptr, (nrows + 1) * 4, kind, ctx->main));
      if (nnz > 0) {
        CP_CUDA(cudaMemcpyAsync(m->col, col, nnz * 4, kind, ctx->main));
        CP_CUDA(cudaMemcpyAsync(m->val, val, nnz * 8, kind, ctx->main));
      }
      csr_validate(ctx, m);  // synchronises the main stream
    } catch (...) {
      dfree_async(m->rowptr, ctx->main);
      dfree_async(m->col, ctx->main);
      dfree_async(m->val, ctx->main);
      cudaStreamSynchronize(ctx->main);
      delete m;
      throw;
    }
    *out = m;
  });
}

cp_status cp_mat_free(cp_mat* m) {
  return guard([&] {
    if (!m) return;
    use_device(m->ctx);
    cudaStreamSynchronize(m->ctx->main);
    cudaStreamSynchronize(m->ctx->side);
    free_formats(m);
    dfree_async(m->rowptr, m->ctx->main);
    dfree_async(m->col, m->ctx->main);
    dfree_async(m->val, m->ctx->main);
    cudaStreamSynchronize(m->ctx->main);
    delete m;
  });
}

cp_status cp_mat_reset(cp_mat* m) {
  return guard([&] {
    CP_REQUIRE(m, CP_ERR_INVALID, "NULL argument");
    use_device(m->ctx);
    CP_CUDA(cudaStreamSynchronize(m->ctx->main));
    CP_CUDA(cudaStreamSynchronize(m->ctx->side));
    std::lock_guard<std::mutex> lock(m->mu);
    free_formats(m);
    m->has_features = false;
    m->batch_tpr_gen = 0;
  });
}

cp_status cp_features(cp_ctx* ctx, cp_mat* m, double* out15) {
  return guard([&] {
    CP_REQUIRE(ctx && m && out15, CP_ERR_INVALID, "NULL argument");
    use_device(ctx);
    compute_features(ctx, m, ctx->main, out15);
  });
}

cp_status cp_convert(cp_ctx* ctx, cp_mat* m, const cp_config* cfg) {
  return guard([&] {
    CP_REQUIRE(ctx && m && cfg, CP_ERR_INVALID, "NULL argument");
    use_device(ctx);
    ensure_format(ctx, m, *cfg, ctx->main);
    CP_CUDA(cudaStreamSynchronize(ctx->main));
  });
}

cp_status cp_format_dims(cp_ctx* ctx, cp_mat* m, const cp_config* cfg, int64_t dims[4]) {
  return guard([&] {
    CP_REQUIRE(ctx && m && cfg && dims, CP_ERR_INVALID, "NULL argument");
    use_device(ctx);
    ensure_format(ctx, m, *cfg, ctx->main);
    format_dims(m, *cfg, dims);
  });
}

cp_status cp_format_export(cp_ctx* ctx, cp_mat* m, const cp_config* cfg, int32_t array_id,
                           void* dst, int64_t capacity, int64_t* bytes) {
  return guard([&] {
    CP_REQUIRE(ctx && m && cfg && dst && bytes, CP_ERR_INVALID, "NULL argument");
    use_device(ctx);
    ensure_format(ctx, m, *cfg, ctx->main);
    format_export(m, *cfg, array_id, dst, capacity, bytes, ctx->main);
  });
}

cp_status cp_spmv(cp_ctx* ctx, cp_mat* m, const cp_config* cfg, int32_t dtype, double alpha,
                  const void* x, double beta, void* y) {
  return guard([&] {
    CP_REQUIRE(ctx && m && x && y, CP_ERR_INVALID, "NULL argument");
    CP_REQUIRE(dtype == CP_DTYPE_F64 || dtype == CP_DTYPE_F32, CP_ERR_INVALID, "bad dtype %d",
               dtype);
    use_device(ctx);
    cp_config c;
    cp_config_default(&c);
    if (cfg) c = *cfg;
    ensure_format(ctx, m, c, ctx->main);
    if (dtype == CP_DTYPE_F64) {
      spmv_general<double>(ctx, m, c, alpha, static_cast<const double*>(x), beta,
                           static_cast<double*>(y), ctx->main);
    } else {
      ensure_val32(ctx, m, c, ctx->main);
      spmv_general<float>(ctx, m, c, (float)alpha, static_cast<const float*>(x), (float)beta,
                          static_cast<float*>(y), ctx->main);
    }
  });
}

cp_status cp_solve_cg(cp_ctx* ctx, cp_mat* m, const double* b, double* x,
                      const cp_solve_opts* opts, cp_solve_info* info) {
  return guard([&] {
    CP_REQUIRE(ctx && m && b && x, CP_ERR_INVALID, "NULL argument");
    use_device(ctx);
    solve(ctx, m, b, x, opts, info, false);
  });
}

cp_status cp_solve_gmres(cp_ctx* ctx, cp_mat* m, const double* b, double* x,
                         const cp_solve_opts* opts, cp_solve_info* info) {
  return guard([&] {
    CP_REQUIRE(ctx && m && b && x, CP_ERR_INVALID, "NULL argument");
    use_device(ctx);
    solve(ctx, m, b, x, opts, info, true);
  });
}

cp_status cp_batch_solve(cp_ctx* ctx, int32_t nsys, cp_mat* const* mats, const int32_t* solver,
                         const double* const* b, double* const* x, const cp_solve_opts* opts,
                         int32_t threads, int32_t threads_per_row, cp_solve_info* infos) {
  return guard([&] {
    CP_REQUIRE(ctx, CP_ERR_INVALID, "NULL context");
    use_device(ctx);
    batch_solve(ctx, nsys, mats, solver, b, x, opts, infos, threads, threads_per_row);
  });
}

cp_status cp_inject_side_failure(cp_ctx* ctx, int32_t point) {
  return guard([&] {
    CP_REQUIRE(ctx && point >= -1 && point <= 2, CP_ERR_INVALID, "bad injection point %d", point);
    ctx->inject_side_fail.store(point);
  });
}

cp_status cp_gate_set(cp_ctx* ctx, const cp_gate* gate) {
  return guard([&] {
    CP_REQUIRE(ctx && gate, CP_ERR_INVALID, "NULL argument");
    for (int f = 0; f < CP_NUM_FMT; ++f)
      CP_REQUIRE(std::isfinite(gate->speedup[f]) && std::isfinite(gate->conv_a_ms[f]) &&
                     std::isfinite(gate->conv_b_ms[f]),
                 CP_ERR_INVALID, "gate figures must be finite");
    CP_REQUIRE(gate->spmv_a_ms >= 0.0 && gate->spmv_b_ms >= 0.0 &&
                   gate->spmv_a_ms + gate->spmv_b_ms > 0.0,
               CP_ERR_INVALID, "the default SpMV time fit must be positive");
    CP_REQUIRE(std::isfinite(gate->feat_a_ms) && std::isfinite(gate->feat_b_ms) &&
                   gate->small_rows >= 0,
               CP_ERR_INVALID, "feature-cost figures must be finite, small_rows >= 0");
    ctx->gate = *gate;
  });
}

static void check_neighbours(int32_t count, int32_t k, const double* mu, const double* sd,
                             const float* z, const float* speedup) {
  CP_REQUIRE(count >= 1 && k >= 1, CP_ERR_INVALID, "count and k must be >= 1");
  CP_REQUIRE(mu && sd && z && speedup, CP_ERR_INVALID, "NULL argument");
  for (int i = 0; i < 15; ++i)
    CP_REQUIRE(std::isfinite(mu[i]) && sd[i] > 0.0 && std::isfinite(sd[i]), CP_ERR_INVALID,
               "mu must be finite and sd positive");
}

cp_status cp_gate_knn_speedup(int32_t count, int32_t k, const double* mu, const double* sd,
                              const float* z, const float* speedup, const double* features,
                              int32_t fmt, double* out) {
  return guard([&] {
    check_neighbours(count, k, mu, sd, z, speedup);
    CP_REQUIRE(features && out, CP_ERR_INVALID, "NULL argument");
    CP_REQUIRE(fmt >= 0 && fmt < CP_NUM_FMT, CP_ERR_INVALID, "fmt must be in 0..%d",
               CP_NUM_FMT - 1);
    *out = gate_knn_speedup(count, k, mu, sd, z, speedup, features, fmt);
  });
}

cp_status cp_gate_set_neighbours(cp_ctx* ctx, int32_t count, int32_t k, const double* mu,
                                 const double* sd, const float* z, const float* speedup) {
  return guard([&] {
    CP_REQUIRE(ctx, CP_ERR_INVALID, "NULL context");
    cp_ctx::GateNeighbours nb;
    if (count != 0) {
      check_neighbours(count, k, mu, sd, z, speedup);
      nb.count = count;
      nb.k = k < count ? k : count;
      std::memcpy(nb.mu, mu, sizeof(nb.mu));
      std::memcpy(nb.sd, sd, sizeof(nb.sd));
      nb.z.assign(z, z + (int64_t)count * 15);
      nb.speedup.assign(speedup, speedup + (int64_t)count * CP_NUM_FMT);
    }
    std::lock_guard<std::mutex> lock(ctx->gate_mu);
    ctx->gate_nb = std::move(nb);
  });
}

int32_t cp_gate_decide(const cp_gate* gate, int32_t fmt, int64_t nnz, int32_t iters, double res0,
                       double res, double target, double* remaining, double* cost_spmvs) {
  if (!gate) return 1;
  return gate_decide(*gate, fmt, nnz, iters, res0, res, target, remaining, cost_spmvs);
}

double cp_gate_payback(const cp_gate* gate, int32_t fmt, int64_t nnz) {
  if (!gate) return 0.0;
  return gate_payback(*gate, fmt, nnz);
}

cp_status cp_batch_tune(cp_ctx* ctx, int32_t nsys, cp_mat* const* mats, const int32_t* solver,
                        const double* const* b, const cp_solve_opts* opts,
                        int32_t* best_threads, int32_t* best_threads_per_row,
                        int32_t* best_order, float* ms, float* ms_order) {
  return guard([&] {
    CP_REQUIRE(ctx, CP_ERR_INVALID, "NULL context");
    use_device(ctx);
    const BatchSchedule best = batch_tune(ctx, nsys, mats, solver, b, opts, ms, ms_order);
    if (best_threads) *best_threads = best.threads;
    if (best_threads_per_row) *best_threads_per_row = best.tpv;
    if (best_order) *best_order = best.order;
  });
}

cp_status cp_batch_tpr(cp_ctx* ctx, cp_mat* m, int32_t* tpr) {
  return guard([&] {
    CP_REQUIRE(ctx && m && tpr, CP_ERR_INVALID, "NULL argument");
    use_device(ctx);
    *tpr = batch_tpr_of(ctx, m, ctx->main);
  });
}

cp_status cp_batch_schedule(cp_ctx* ctx, int64_t mean_rows, int32_t has_gmres, int32_t* threads,
                            int32_t* threads_per_row, int32_t* order) {
  return guard([&] {
    CP_REQUIRE(ctx && threads && threads_per_row, CP_ERR_INVALID, "NULL argument");
    const BatchSchedule sc = batch_schedule(ctx, mean_rows, has_gmres != 0);
    *threads = sc.threads;
    *threads_per_row = sc.tpv;
    if (order) *order = sc.order;
  });
}

int64_t cp_mlp_nparams(int32_t d, int32_t h1, int32_t h2, int32_t k) {
  return (int64_t)h1 * d + h1 + (int64_t)h2 * h1 + h2 + (int64_t)k * h2 + k;
}

int64_t cp_mlp_scratch_floats(int64_t N, int32_t d, int32_t h1, int32_t h2, int32_t k) {
  return scratch_floats_api(N, d, h1, h2, k);
}

cp_status cp_mlp_forward(cp_ctx* ctx, int64_t N, int32_t d, int32_t h1, int32_t h2, int32_t k,
                         const float* params, const float* X, float* logits, float* scratch) {
  return guard([&] {
    CP_REQUIRE(ctx && params && X && logits && scratch && N >= 1, CP_ERR_INVALID, "bad argument");
    use_device(ctx);
    mlp_forward(ctx, N, MlpDims{d, h1, h2, k}, params, X, logits, scratch, ctx->main);
  });
}

cp_status cp_mlp_loss_grad(cp_ctx* ctx, int64_t N, int32_t d, int32_t h1, int32_t h2, int32_t k,
                           const float* params, const float* X, const int32_t* labels,
                           float* loss, float* grad, float* scratch) {
  return guard([&] {
    CP_REQUIRE(ctx && params && X && labels && loss && grad && scratch && N >= 1, CP_ERR_INVALID,
               "bad argument");
    use_device(ctx);
    mlp_loss_grad(ctx, N, MlpDims{d, h1, h2, k}, params, X, labels, nullptr, loss, grad,
                  scratch, ctx->main);
  });
}

cp_status cp_mlp_loss_grad_soft(cp_ctx* ctx, int64_t N, int32_t d, int32_t h1, int32_t h2,
                                int32_t k, const float* params, const float* X,
                                const float* targets, float* loss, float* grad, float* scratch) {
  return guard([&] {
    CP_REQUIRE(ctx && params && X && targets && loss && grad && scratch && N >= 1,
               CP_ERR_INVALID, "bad argument");
    use_device(ctx);
    mlp_loss_grad(ctx, N, MlpDims{d, h1, h2, k}, params, X, nullptr, targets, loss, grad,
                  scratch, ctx->main);
  });
}

cp_status cp_adam_step(cp_ctx* ctx, int64_t nparams, float* params, const float* grad, float* m,
                       float* v, int32_t t, float lr, float beta1, float beta2, float eps) {
  return guard([&] {
    CP_REQUIRE(ctx && params && grad && m && v && nparams >= 1, CP_ERR_INVALID, "bad argument");
    use_device(ctx);
    adam_step(ctx, nparams, params, grad, m, v, t, lr, beta1, beta2, eps, ctx->main);
  });
}

cp_status cp_model_load(cp_ctx* ctx, int32_t stage, int32_t h1, int32_t h2, int32_t k,
                        const float* params, const float* mu, const float* sd) {
  return guard([&] {
    CP_REQUIRE(ctx && params && mu && sd, CP_ERR_INVALID, "NULL argument");
    use_device(ctx);
    model_install(ctx, stage, h1, h2, k, params, mu, sd, ctx->main);
  });
}

cp_status cp_model_get(cp_ctx* ctx, int32_t stage, int32_t dims[4], float* params,
                       int64_t capacity, float* mu, float* sd) {
  return guard([&] {
    CP_REQUIRE(ctx && dims && stage >= 0 && stage < CP_NUM_STAGES, CP_ERR_INVALID, "bad argument");
    use_device(ctx);
    std::lock_guard<std::mutex> lock(ctx->model_mu);
    const ModelSlot& s = ctx->models[stage];
    CP_REQUIRE(s.loaded, CP_ERR_INVALID, "stage %d has no model", stage);
    dims[0] = 15;
    dims[1] = s.h1;
    dims[2] = s.h2;
    dims[3] = s.k;
    const int64_t np = cp_mlp_nparams(15, s.h1, s.h2, s.k);
    if (params) {
      CP_REQUIRE(capacity >= np, CP_ERR_INVALID, "params needs %lld floats", (long long)np);
      CP_CUDA(cudaMemcpy(params, s.d_params, np * 4, cudaMemcpyDeviceToHost));
    }
    if (mu) CP_CUDA(cudaMemcpy(mu, s.d_mu, 15 * 4, cudaMemcpyDeviceToHost));
    if (sd) CP_CUDA(cudaMemcpy(sd, s.d_sd, 15 * 4, cudaMemcpyDeviceToHost));
  });
}

cp_status cp_model_train(cp_ctx* ctx, int32_t stage, int64_t N, const double* F,
                         const int32_t* labels, int32_t h1, int32_t h2, int32_t k,
                         int32_t epochs, float lr, uint64_t seed, float* final_loss) {
  return guard([&] {
    CP_REQUIRE(ctx && F && labels && epochs >= 0, CP_ERR_INVALID, "bad argument");
    use_device(ctx);
    model_train(ctx, stage, N, F, labels, nullptr, h1, h2, k, epochs, lr, seed, final_loss);
  });
}

cp_status cp_model_train_soft(cp_ctx* ctx, int32_t stage, int64_t N, const double* F,
                              const float* targets, int32_t h1, int32_t h2, int32_t k,
                              int32_t epochs, float lr, uint64_t seed, float* final_loss) {
  return guard([&] {
    CP_REQUIRE(ctx && F && targets && epochs >= 0, CP_ERR_INVALID, "bad argument");
    use_device(ctx);
    model_train(ctx, stage, N, F, nullptr, targets, h1, h2, k, epochs, lr, seed, final_loss);
  });
}

cp_status cp_predict_stage(cp_ctx* ctx, int32_t stage, const double* features15,
                           float* logits, int32_t* pick) {
  return guard([&] {
    CP_REQUIRE(ctx && features15, CP_ERR_INVALID, "NULL argument");
    CP_REQUIRE(stage >= 0 && stage < CP_NUM_STAGES, CP_ERR_INVALID, "bad stage %d", stage);
    CP_REQUIRE(stage_classes(ctx, stage) > 0, CP_ERR_INVALID, "stage %d has no model", stage);
    use_device(ctx);
    const int p = infer_stage(ctx, stage, features15, ctx->side, logits);
    if (pick) *pick = p;
  });
}

cp_status cp_predict(cp_ctx* ctx, cp_mat* m, cp_config* out, float* stage_ms) {
  return guard([&] {
    CP_REQUIRE(ctx && m && out, CP_ERR_INVALID, "NULL argument");
    use_device(ctx);
    Channel ch;
    run_cascade(ctx, m, ctx->side, &ch);
    CP_REQUIRE(ch.status == CP_OK, ch.status, "%s", ch.error.c_str());
    cp_config_default(out);
    for (auto& p : ch.published) *out = p.second;
    if (stage_ms) {
      stage_ms[0] = ch.t_features_ms;
      stage_ms[1] = ch.t_predict_ms[0];
      stage_ms[2] = ch.t_predict_ms[1];
      stage_ms[3] = ch.t_predict_ms[2];
    }
  });
}

}  // extern "C"
