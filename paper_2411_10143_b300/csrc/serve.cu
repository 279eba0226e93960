// Continuous-batching solve server.
//
// Requests (a resident matrix, a right-hand side, a solution buffer) arrive at
// any time.  A scheduler thread admits them while their Krylov workspace fits
// the HBM budget and hands work to `lanes` worker threads, each with its own
// context and streams, so several solves run on the device at once:
//  - a request with n <= small_max_n (GMRES: small_max_n_gmres) joins the next
//    batch: a free lane takes
//    every admitted small request (up to max_batch) into one persistent,
//    graph-captured batched launch (cp_batch_solve's kernel);
//  - a larger request gets a lane of its own and runs the asynchronous
//    cascaded solver with FP32 inner solves inside FP64 refinement.
// Requests that arrive while others run are admitted as soon as a lane and
// memory free up.  Every completion records submit / start / done times.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

struct cp_server {
  cp_ctx* parent = nullptr;
  cp_server_opts opts;
  std::vector<cp_ctx*> lane_ctx;
  std::vector<std::thread> workers;
  std::thread scheduler;
  std::mutex mu;
  std::condition_variable cv;       // scheduler wake-up
  std::condition_variable lane_cv;  // worker wake-up
  std::deque<cp_request> pending;   // submitted, not admitted
  struct Job {
    bool batch = false;
    std::vector<cp_request> reqs;
    std::vector<double> t_submit;
    double t_admit = 0.0;
    int64_t bytes = 0;
  };
  std::vector<std::deque<Job>> lane_jobs;
  std::vector<int> lane_busy;
  std::atomic<int> busy{0};  // lanes holding a job (read by the lanes' solves)
  std::deque<double> pending_submit;  // submit time of every pending request
  std::vector<cp_result> done;
  int64_t in_use_bytes = 0;
  int64_t inflight = 0;
  bool stop = false;
  std::chrono::steady_clock::time_point t0;
  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace cp {

// Whether a request joins a batch (else it gets a lane of its own).
static bool batched(const cp_request& r, const cp_server_opts& o) {
  const int64_t lim = r.solver == 1 ? std::min(o.small_max_n, o.small_max_n_gmres) : o.small_max_n;
  return r.mat->nrows <= lim;
}

// Device workspace a request needs while it runs (its matrix is already resident).
static int64_t request_bytes(const cp_request& r, const cp_server_opts& o) {
  const int64_t n = r.mat->nrows;
  const int64_t m = o.restart > 0 ? o.restart : 30;
  if (batched(r, o)) return n * 8 + (r.solver == 0 ? 4 : m + 2) * n * 4;
  // full-GPU solver: FP64 refinement vectors + FP32 inner (CG 3n, GMRES (m+2)n)
  return 4 * n * 8 + (r.solver == 0 ? 3 : m + 2) * n * 4 + n * 4 + r.mat->nnz * 4;
}

static void run_job(cp_server* S, int lane, cp_server::Job& job) {
  cp_ctx* ctx = S->lane_ctx[lane];
  const double t_start = S->now_ms();
  std::vector<cp_result> res(job.reqs.size());
  cp_solve_opts o;
  cp_solve_opts_default(&o);
  o.tol = S->opts.tol;
  o.inner_tol = S->opts.inner_tol;
  o.ir_theta = S->opts.ir_theta;
  o.restart = S->opts.restart > 0 ? S->opts.restart : 30;
  o.precision = CP_PREC_FP32_IR;
  o.maxit = S->opts.maxit > 0 ? S->opts.maxit : 100000;
  try {
    CP_CUDA(cudaSetDevice(ctx->device));
    if (job.batch) {
      const int nb = (int)job.reqs.size();
      std::vector<cp_mat*> mats(nb);
      std::vector<int32_t> solver(nb);
      std::vector<const double*> b(nb);
      std::vector<double*> x(nb);
      std::vector<cp_solve_info> infos(nb);
      for (int i = 0; i < nb; ++i) {
        mats[i] = job.reqs[i].mat;
        solver[i] = job.reqs[i].solver;
        b[i] = job.reqs[i].b;
        x[i] = job.reqs[i].x;
      }
      cp_status st = CP_OK;
      try {
        batch_solve(ctx, nb, mats.data(), solver.data(), b.data(), x.data(), &o, infos.data(), 0,
                    0);
      } catch (const Error& e) {
        st = e.status;
      }
      for (int i = 0; i < nb; ++i) {
        res[i].status = infos[i].status != CP_OK ? infos[i].status : st == CP_OK ? CP_OK : st;
        res[i].iters = infos[i].iters;
        res[i].relres_true = infos[i].relres_true;
        res[i].batched = 1;
      }
    } else {
      const cp_request& r = job.reqs[0];
      o.mode = S->opts.mode;
      // lanes run concurrently and cooperative grids sized for the whole
      // device must not share it: the solve takes the persistent kernels only
      // while this is the one busy lane, and a running one returns at its next
      // iteration boundary once another lane gets work (ctx->lanes_busy)
      o.iteration_kernel = 0;
      cp_solve_info info;
      std::memset(&info, 0, sizeof(info));
      cp_status st = CP_OK;
      try {
        solve(ctx, r.mat, r.b, r.x, &o, &info, r.solver == 1);
      } catch (const Error& e) {
        st = e.status;
      }
      res[0].status = st;
      res[0].iters = info.iters;
      res[0].relres_true = info.relres_true;
      res[0].batched = 0;
    }
  } catch (const Error& e) {
    for (auto& q : res) q.status = e.status;
  }
  const double t_done = S->now_ms();
  std::lock_guard<std::mutex> lock(S->mu);
  for (size_t i = 0; i < job.reqs.size(); ++i) {
    res[i].id = job.reqs[i].id;
    res[i].t_submit_ms = job.t_submit[i];
    res[i].t_start_ms = t_start;
    res[i].t_done_ms = t_done;
    res[i].lane = lane;
    S->done.push_back(res[i]);
  }
  S->in_use_bytes -= job.bytes;
  S->inflight -= (int64_t)job.reqs.size();
  S->lane_busy[lane] = 0;
  S->busy.fetch_sub(1, std::memory_order_acq_rel);
  S->cv.notify_all();
}

static void worker_loop(cp_server* S, int lane) {
  for (;;) {
    cp_server::Job job;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->lane_cv.wait(lock, [&] { return S->stop || !S->lane_jobs[lane].empty(); });
      if (S->lane_jobs[lane].empty()) return;  // stop requested and nothing queued
      job = std::move(S->lane_jobs[lane].front());
      S->lane_jobs[lane].pop_front();
    }
    run_job(S, lane, job);
  }
}

// Admission and placement: runs whenever a request arrives or a lane frees up.
static void scheduler_loop(cp_server* S) {
  std::unique_lock<std::mutex> lock(S->mu);
  const cp_server_opts& o = S->opts;
  for (;;) {
    S->cv.wait(lock, [&] {
      if (S->stop) return true;
      if (S->pending.empty()) return false;
      for (size_t l = 0; l < S->lane_busy.size(); ++l)
        if (!S->lane_busy[l]) return true;
      return false;
    });
    if (S->stop) return;
    int lane = -1;
    for (size_t l = 0; l < S->lane_busy.size(); ++l)
      if (!S->lane_busy[l]) {
        lane = (int)l;
        break;
      }
    if (lane < 0 || S->pending.empty()) continue;
    cp_server::Job job;
    job.t_admit = S->now_ms();
    const cp_request& head = S->pending.front();
    if (!batched(head, o)) {
      const int64_t need = request_bytes(head, o);
      if (S->in_use_bytes + need > o.mem_budget && S->in_use_bytes > 0) {
        // wait for memory to free up (a running job will notify)
        S->cv.wait(lock, [&] { return S->stop || S->in_use_bytes + need <= o.mem_budget ||
                                      S->in_use_bytes == 0; });
        if (S->stop) return;
        continue;
      }
      job.reqs.push_back(head);
      job.t_submit.push_back(S->pending_submit.front());
      job.bytes = need;
      S->pending.pop_front();
      S->pending_submit.pop_front();
    } else {
      // every admitted small request, in arrival order, up to max_batch and budget;
      // large ones stay queued in order
      job.batch = true;
      std::deque<cp_request> keep;
      std::deque<double> keep_t;
      while (!S->pending.empty()) {
        cp_request r = S->pending.front();
        const double ts = S->pending_submit.front();
        S->pending.pop_front();
        S->pending_submit.pop_front();
        const int64_t need = request_bytes(r, o);
        if (batched(r, o) && (int)job.reqs.size() < o.max_batch &&
            S->in_use_bytes + job.bytes + need <= o.mem_budget) {
          job.reqs.push_back(r);
          job.t_submit.push_back(ts);
          job.bytes += need;
        } else {
          keep.push_back(r);
          keep_t.push_back(ts);
        }
      }
      S->pending.swap(keep);
      S->pending_submit.swap(keep_t);
      if (job.reqs.empty()) {
        S->cv.wait(lock, [&] { return S->stop || S->in_use_bytes == 0; });
        if (S->stop) return;
        continue;
      }
    }
    S->in_use_bytes += job.bytes;
    S->lane_busy[lane] = 1;
    S->busy.fetch_add(1, std::memory_order_acq_rel);  // before the job can start
    S->lane_jobs[lane].push_back(std::move(job));
    S->lane_cv.notify_all();
  }
}

}  // namespace cp

using namespace cp;

extern "C" {

void cp_server_opts_default(cp_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->inner_tol = 1e-5;
  o->restart = 30;
  o->maxit = 100000;
  o->small_max_n = 32768;
  o->small_max_n_gmres = 8192;
  o->max_batch = 256;
  o->lanes = 4;
  o->mem_budget = int64_t(16) << 30;
  o->mode = CP_MODE_ASYNC;
  o->ir_theta = 0.5;
}

cp_status cp_server_create(cp_ctx* ctx, const cp_server_opts* opts, cp_server** out) {
  try {
    CP_REQUIRE(ctx && out, CP_ERR_INVALID, "NULL argument");
    *out = nullptr;
    cp_server* S = new cp_server();
    cp_server_opts_default(&S->opts);
    if (opts) S->opts = *opts;
    CP_REQUIRE(S->opts.lanes >= 1 && S->opts.lanes <= 32 && S->opts.max_batch >= 1 &&
                   S->opts.restart >= 1 && S->opts.restart <= 32 && S->opts.mem_budget > 0 &&
                   S->opts.ir_theta >= 0.0 && S->opts.ir_theta < 1.0,
               CP_ERR_INVALID, "bad server options");
    S->parent = ctx;
    // the lanes share this process's loaded kernels: load them once, before the
    // first request's time starts
    {
      const cp_status ws = cp_warmup(ctx);
      if (ws != CP_OK) {
        delete S;
        return ws;
      }
    }
    S->t0 = std::chrono::steady_clock::now();
    const int L = S->opts.lanes;
    S->lane_jobs.resize(L);
    S->lane_busy.assign(L, 0);
    for (int l = 0; l < L; ++l) {
      cp_ctx* c = nullptr;
      cp_status st = cp_create(&c, ctx->device, nullptr, nullptr);
      if (st != CP_OK) {
        for (auto* q : S->lane_ctx) cp_destroy(q);
        delete S;
        return st;
      }
      // every lane shares the parent's cascade models
      for (int k = 0; k < CP_NUM_STAGES; ++k) {
        const ModelSlot& ms = ctx->models[k];
        if (ms.loaded) model_install(c, k, ms.h1, ms.h2, ms.k, ms.d_params, ms.d_mu, ms.d_sd,
                                     c->main, ms.gen);
      }
      c->lanes_busy = &S->busy;
      S->lane_ctx.push_back(c);
    }
    for (int l = 0; l < L; ++l) S->workers.emplace_back(worker_loop, S, l);
    S->scheduler = std::thread(scheduler_loop, S);
    *out = S;
    return CP_OK;
  } catch (const Error& e) {
    return e.status;
  } catch (...) {
    return CP_ERR_CUDA;
  }
}

cp_status cp_server_submit(cp_server* S, const cp_request* r) {
  try {
    CP_REQUIRE(S && r && r->mat && r->b && r->x, CP_ERR_INVALID, "NULL argument");
    CP_REQUIRE(r->mat->nrows == r->mat->ncols && (r->solver == 0 || r->solver == 1),
               CP_ERR_INVALID, "bad request");
    std::lock_guard<std::mutex> lock(S->mu);
    S->pending.push_back(*r);
    S->pending_submit.push_back(S->now_ms());
    S->inflight += 1;
    S->cv.notify_all();
    return CP_OK;
  } catch (const Error& e) {
    return e.status;
  }
}

cp_status cp_server_poll(cp_server* S, cp_result* out, int32_t capacity, int32_t* count) {
  if (!S || !count || (capacity > 0 && !out)) return CP_ERR_INVALID;
  std::lock_guard<std::mutex> lock(S->mu);
  const int32_t k = (int32_t)std::min<size_t>(S->done.size(), (size_t)capacity);
  for (int32_t i = 0; i < k; ++i) out[i] = S->done[i];
  S->done.erase(S->done.begin(), S->done.begin() + k);
  *count = k;
  return CP_OK;
}

cp_status cp_server_drain(cp_server* S, double timeout_s) {
  if (!S) return CP_ERR_INVALID;
  std::unique_lock<std::mutex> lock(S->mu);
  const bool ok = S->cv.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                 [&] { return S->inflight == 0; });
  return ok ? CP_OK : CP_ERR_TIMEOUT;
}

cp_status cp_server_destroy(cp_server* S) {
  if (!S) return CP_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  S->lane_cv.notify_all();
  if (S->scheduler.joinable()) S->scheduler.join();
  for (auto& w : S->workers)
    if (w.joinable()) w.join();
  for (auto* c : S->lane_ctx) cp_destroy(c);
  delete S;
  return CP_OK;
}

}  // extern "C"
