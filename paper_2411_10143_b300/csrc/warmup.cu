// cp_warmup: one pass over the kernels a solve can launch, on a small internal
// system, so that no solve pays their one-time costs.  The CUDA runtime loads a
// kernel at its first launch in the process (lazy module loading); the first
// launch of the persistent kernels and of the conversion kernels was measured
// to add tens of milliseconds to the first asynchronous solve of a process (an
// 86 ms first GMRES(30) solve of convection-diffusion 96^3 against 59 ms for
// the next), inside that solve's time-to-solution.
#include <vector>

#include "internal.cuh"

namespace {

struct Buf {
  void* p = nullptr;
  ~Buf() {
    if (p) cudaFree(p);
  }
};

void check(cp_status st) {
  // a warm-up solve may stop at its iteration limit; anything else is an error
  if (st != CP_OK && st != CP_ERR_NOT_CONVERGED) throw cp::Error{st};
}

}  // namespace

extern "C" cp_status cp_warmup(cp_ctx* ctx) {
  cp_mat* m = nullptr;
  try {
    CP_REQUIRE(ctx, CP_ERR_INVALID, "NULL argument");
    // 3D 7-point Poisson on a 10^3 grid (1,000 rows): symmetric positive
    // definite (CG) with seven diagonals (DIA), and more than one block of rows
    const int k = 10, n = k * k * k;
    std::vector<int32_t> rp(1, 0), ci;
    std::vector<double> va;
    for (int z = 0; z < k; ++z)
      for (int y = 0; y < k; ++y)
        for (int x = 0; x < k; ++x) {
          const int i = (z * k + y) * k + x;
          const int nb[7] = {i - k * k, i - k, i - 1, i, i + 1, i + k, i + k * k};
          const bool in[7] = {z > 0, y > 0, x > 0, true, x < k - 1, y < k - 1, z < k - 1};
          for (int q = 0; q < 7; ++q) {
            if (!in[q]) continue;
            ci.push_back(nb[q]);
            va.push_back(q == 3 ? 6.0 : -1.0);
          }
          rp.push_back((int32_t)ci.size());
        }
    check(cp_csr_load(ctx, n, n, (int64_t)ci.size(), rp.data(), ci.data(), va.data(), 0, &m));
    Buf b, x, bf, xf;
    CP_CUDA(cudaMalloc(&b.p, n * sizeof(double)));
    CP_CUDA(cudaMalloc(&x.p, n * sizeof(double)));
    CP_CUDA(cudaMalloc(&bf.p, n * sizeof(float)));
    CP_CUDA(cudaMalloc(&xf.p, n * sizeof(float)));
    const std::vector<double> ones(n, 1.0);
    CP_CUDA(cudaMemcpy(b.p, ones.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    CP_CUDA(cudaMemset(bf.p, 0, n * sizeof(float)));
    double* bd = static_cast<double*>(b.p);
    double* xd = static_cast<double*>(x.p);

    // features and, where models are installed, the cascade's inference
    double feat[15];
    check(cp_features(ctx, m, feat));
    cp_config pred;
    bool have_models = true;
    for (int s = CP_STAGE_FORMAT; s <= CP_STAGE_SELL_SIGMA; ++s)  // the cascade's stages
      have_models = have_models && ctx->models[s].loaded;
    if (have_models) check(cp_predict(ctx, m, &pred, nullptr));

    std::vector<cp_config> cfgs;
    auto add = [&](int fmt, int algo, int tpv, int sigma) {
      cp_config c;
      cp_config_default(&c);
      c.fmt = fmt;
      c.algo = algo;
      c.tpv = tpv;
      c.sell_sigma = sigma;
      cfgs.push_back(c);
    };
    add(CP_FMT_CSR, CP_ALGO_SCALAR, 8, 1);
    for (int tpv : {2, 4, 8, 16, 32}) add(CP_FMT_CSR, CP_ALGO_VECTOR, tpv, 1);
    add(CP_FMT_CSR, CP_ALGO_MERGE, 8, 1);
    add(CP_FMT_COO, CP_ALGO_SCALAR, 8, 1);
    add(CP_FMT_ELL, CP_ALGO_SCALAR, 8, 1);
    for (int sigma : {1, 32, 1024, 8192}) add(CP_FMT_SELL, CP_ALGO_SCALAR, 8, sigma);
    add(CP_FMT_HYB, CP_ALGO_SCALAR, 8, 1);
    add(CP_FMT_HYB, CP_ALGO_SCALAR, 8, 1);
    cfgs.back().hyb_k = 3;  // rows longer than 3: a COO part (the persistent tail variants)
    add(CP_FMT_DIA, CP_ALGO_SCALAR, 8, 1);

    cp_solve_opts o;
    cp_solve_opts_default(&o);
    o.tol = 1e-6;
    o.maxit = 40;
    o.restart = 8;
    o.inner_tol = 1e-3;
    o.max_outer = 2;
    for (const cp_config& c : cfgs) {
      check(cp_convert(ctx, m, &c));
      check(cp_spmv(ctx, m, &c, CP_DTYPE_F64, 1.0, bd, 0.0, xd));
      check(cp_spmv(ctx, m, &c, CP_DTYPE_F32, 1.0, bf.p, 0.0, xf.p));
      o.force = &c;
      for (int prec : {CP_PREC_FP64, CP_PREC_FP32_IR})
        for (int kernel : {0, 1}) {
          o.precision = prec;
          o.iteration_kernel = kernel;
          for (int orth : {0, 1}) {
            o.gmres_orth = orth;
            CP_CUDA(cudaMemset(xd, 0, n * sizeof(double)));
            check(cp_solve_gmres(ctx, m, bd, xd, &o, nullptr));
          }
          CP_CUDA(cudaMemset(xd, 0, n * sizeof(double)));
          check(cp_solve_cg(ctx, m, bd, xd, &o, nullptr));
        }
    }
    // the asynchronous path: side thread, prediction and switching
    o.force = nullptr;
    o.precision = CP_PREC_FP64;
    o.iteration_kernel = 0;
    o.gmres_orth = 0;
    o.mode = CP_MODE_ASYNC;
    check(cp_mat_reset(m));
    CP_CUDA(cudaMemset(xd, 0, n * sizeof(double)));
    check(cp_solve_cg(ctx, m, bd, xd, &o, nullptr));
    check(cp_mat_reset(m));
    CP_CUDA(cudaMemset(xd, 0, n * sizeof(double)));
    check(cp_solve_gmres(ctx, m, bd, xd, &o, nullptr));
    CP_CUDA(cudaDeviceSynchronize());
    check(cp_mat_free(m));
    return CP_OK;
  } catch (const cp::Error& e) {
    if (m) cp_mat_free(m);
    return e.status;
  } catch (...) {
    if (m) cp_mat_free(m);
    return CP_ERR_CUDA;
  }
}

// ------------------------------------------------------------------ FP64 FMA rate
// The denominator of the FP64-pipe roofline: independent FMA chains, eight per
// thread, on every SM at full occupancy.  The multiplier and addend are kernel
// arguments, so the compiler can neither fold nor shorten a chain; the final
// values are stored only if a condition no finite input meets holds.
namespace {

constexpr int kRateChains = 8;

__global__ void __launch_bounds__(256) k_dfma_rate(int iters, double mul, double add,
                                                   double* sink) {
  double a[kRateChains];
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) a[c] = 1.0 + 1e-3 * c + 1e-9 * threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) a[c] = fma(a[c], mul, add);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kRateChains; ++c) s += a[c];
  if (s == -1.0) sink[blockIdx.x] = s;  // never true for the inputs used
}

}  // namespace

extern "C" cp_status cp_fp64_fma_rate(cp_ctx* ctx, double* fma_per_s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double* sink = nullptr;
  try {
    CP_REQUIRE(ctx && fma_per_s, CP_ERR_INVALID, "NULL argument");
    CP_CUDA(cudaSetDevice(ctx->device));
    int sms = 0;
    CP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int block = 256, grid = sms * 8, iters = 4096;  // 2,048 threads per SM
    CP_CUDA(cudaMalloc(&sink, sizeof(double) * grid));
    CP_CUDA(cudaEventCreate(&e0));
    CP_CUDA(cudaEventCreate(&e1));
    cudaStream_t s = ctx->main;
    float best = 1e30f;
    for (int rep = 0; rep < 6; ++rep) {  // the first launch loads the kernel: not kept
      CP_CUDA(cudaEventRecord(e0, s));
      CP_LAUNCH(ctx, k_dfma_rate, grid, block, 0, s, iters, 0.9999999, 1e-7, sink);
      CP_CUDA(cudaEventRecord(e1, s));
      CP_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      CP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms < best) best = ms;
    }
    *fma_per_s = (double)grid * block * iters * kRateChains / (best * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return CP_OK;
  } catch (const cp::Error& e) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    return e.status;
  }
}
