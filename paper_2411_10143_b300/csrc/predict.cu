// Cascaded prediction (Sec. III-C-1, Fig. 5) and its classifiers.
//
// Every cascade stage is a small MLP d -> h1 -> h2 -> k (ReLU) on the
// standardised log-features z_j = (log(1 + f_j) - mu_j) / sd_j of Table IV.
// The paper trains LightGBM models with AutoGluon and compiles them to C so
// that inference costs microseconds (Sec. III-C-2, Table V); here inference is
// one GPU block on the side stream, and training runs on the GPU with the
// forward / backward / Adam kernels below.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <thread>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.cuh"
#include "persist.cuh"

namespace cp {

constexpr int kFeat = 15;
constexpr int kMaxHidden = 64;
constexpr int kMaxClass = 8;

// Scratch layout (floats): A1[N][h1], A2[N][h2], Z[N][k], G1[N][h1], G2[N][h2],
// G3[N][k], L[N]
static int64_t scratch_floats(int64_t N, const MlpDims& D) {
  return N * (2 * (int64_t)D.h1 + 2 * (int64_t)D.h2 + 2 * (int64_t)D.k + 1);
}

// ------------------------------------------------------------------ kernels
// Thread per sample: the forward pass, keeping both hidden activations.
__global__ void k_mlp_fwd(int64_t N, MlpDims D, const float* __restrict__ P,
                          const float* __restrict__ X, float* __restrict__ A1,
                          float* __restrict__ A2, float* __restrict__ Z) {
  const float* W1 = P;
  const float* b1 = W1 + D.h1 * D.d;
  const float* W2 = b1 + D.h1;
  const float* b2 = W2 + D.h2 * D.h1;
  const float* W3 = b2 + D.h2;
  const float* b3 = W3 + D.k * D.h2;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N;
       s += (int64_t)gridDim.x * blockDim.x) {
    const float* x = X + s * D.d;
    float* a1 = A1 + s * D.h1;
    float* a2 = A2 + s * D.h2;
    for (int o = 0; o < D.h1; ++o) {
      float acc = b1[o];
      for (int i = 0; i < D.d; ++i) acc = fmaf(W1[o * D.d + i], x[i], acc);
      a1[o] = acc > 0.f ? acc : 0.f;
    }
    for (int o = 0; o < D.h2; ++o) {
      float acc = b2[o];
      for (int i = 0; i < D.h1; ++i) acc = fmaf(W2[o * D.h1 + i], a1[i], acc);
      a2[o] = acc > 0.f ? acc : 0.f;
    }
    for (int o = 0; o < D.k; ++o) {
      float acc = b3[o];
      for (int i = 0; i < D.h2; ++i) acc = fmaf(W3[o * D.h2 + i], a2[i], acc);
      Z[s * D.k + o] = acc;
    }
  }
}

// Thread per sample: loss and the output / hidden deltas of softmax
// cross-entropy averaged over the batch.  The target of sample s is the class
// lab[s] (Q = NULL), or the distribution Q[s][0..k) (soft targets, rows summing
// to 1): loss = logsumexp(z) - sum_c Q_c z_c, dloss/dz = softmax(z) - Q.
__global__ void k_mlp_bwd(int64_t N, MlpDims D, const float* __restrict__ P,
                          const int32_t* __restrict__ lab, const float* __restrict__ Q,
                          const float* __restrict__ A1, const float* __restrict__ A2,
                          const float* __restrict__ Z, float* __restrict__ G1,
                          float* __restrict__ G2, float* __restrict__ G3, float* __restrict__ L) {
  const float* W2 = P + D.h1 * D.d + D.h1;
  const float* W3 = W2 + D.h2 * D.h1 + D.h2;
  const float invN = 1.f / (float)N;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N;
       s += (int64_t)gridDim.x * blockDim.x) {
    const float* z = Z + s * D.k;
    float zmax = z[0];
    for (int o = 1; o < D.k; ++o) zmax = fmaxf(zmax, z[o]);
    float se = 0.f;
    for (int o = 0; o < D.k; ++o) se += expf(z[o] - zmax);
    const float lse = zmax + logf(se);
    float* g3 = G3 + s * D.k;
    if (Q) {
      const float* q = Q + s * D.k;
      float qz = 0.f;
      for (int o = 0; o < D.k; ++o) qz = fmaf(q[o], z[o], qz);
      L[s] = lse - qz;
      for (int o = 0; o < D.k; ++o) g3[o] = (expf(z[o] - lse) - q[o]) * invN;
    } else {
      const int y = lab[s];
      L[s] = lse - z[y];
      for (int o = 0; o < D.k; ++o) g3[o] = (expf(z[o] - lse) - (o == y ? 1.f : 0.f)) * invN;
    }
    const float* a2 = A2 + s * D.h2;
    float* g2 = G2 + s * D.h2;
    for (int i = 0; i < D.h2; ++i) {
      float acc = 0.f;
      for (int o = 0; o < D.k; ++o) acc = fmaf(W3[o * D.h2 + i], g3[o], acc);
      g2[i] = a2[i] > 0.f ? acc : 0.f;
    }
    const float* a1 = A1 + s * D.h1;
    float* g1 = G1 + s * D.h1;
    for (int i = 0; i < D.h1; ++i) {
      float acc = 0.f;
      for (int o = 0; o < D.h2; ++o) acc = fmaf(W2[o * D.h1 + i], g2[o], acc);
      g1[i] = a1[i] > 0.f ? acc : 0.f;
    }
  }
}

// Thread per parameter: sum of the per-sample contributions in sample order
// (deterministic).
__global__ void k_mlp_grad(int64_t N, MlpDims D, const float* __restrict__ X,
                           const float* __restrict__ A1, const float* __restrict__ A2,
                           const float* __restrict__ G1, const float* __restrict__ G2,
                           const float* __restrict__ G3, float* __restrict__ grad) {
  const int64_t np = D.nparams();
  const int64_t oW1 = 0, ob1 = oW1 + D.h1 * D.d, oW2 = ob1 + D.h1, ob2 = oW2 + D.h2 * D.h1;
  const int64_t oW3 = ob2 + D.h2, ob3 = oW3 + D.k * D.h2;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
       q += (int64_t)gridDim.x * blockDim.x) {
    const float *g, *a;
    int gs, as, go, ai;  // strides and indices
    if (q < ob1) {
      go = (int)(q / D.d); ai = (int)(q % D.d); g = G1; gs = D.h1; a = X; as = D.d;
    } else if (q < oW2) {
      go = (int)(q - ob1); ai = -1; g = G1; gs = D.h1; a = nullptr; as = 0;
    } else if (q < ob2) {
      go = (int)((q - oW2) / D.h1); ai = (int)((q - oW2) % D.h1); g = G2; gs = D.h2; a = A1; as = D.h1;
    } else if (q < oW3) {
      go = (int)(q - ob2); ai = -1; g = G2; gs = D.h2; a = nullptr; as = 0;
    } else if (q < ob3) {
      go = (int)((q - oW3) / D.h2); ai = (int)((q - oW3) % D.h2); g = G3; gs = D.k; a = A2; as = D.h2;
    } else {
      go = (int)(q - ob3); ai = -1; g = G3; gs = D.k; a = nullptr; as = 0;
    }
    float acc = 0.f;
    if (ai >= 0) {
      for (int64_t s = 0; s < N; ++s) acc = fmaf(g[s * gs + go], a[s * as + ai], acc);
    } else {
      for (int64_t s = 0; s < N; ++s) acc += g[s * gs + go];
    }
    grad[q] = acc;
  }
}

__global__ void k_mlp_loss(int64_t N, const float* __restrict__ L, float* loss) {
  __shared__ double red[33];
  double acc = 0.0;
  for (int64_t s = threadIdx.x; s < N; s += blockDim.x) acc += (double)L[s];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) *loss = (float)(acc / (double)N);
}

__global__ void k_adam(int64_t np, float* __restrict__ P, const float* __restrict__ G,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Feature standardisation for training: one block per feature computes the
// mean and population sd of log(1 + f) over the N samples; then every sample is
// standardised (sd = 0 is replaced by 1).
__global__ void k_feat_stats(int64_t N, const double* __restrict__ F, float* __restrict__ mu,
                             float* __restrict__ sd) {
  __shared__ double red[40];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int64_t q = threadIdx.x; q < N; q += blockDim.x) s += log1p(F[q * kFeat + j]);
  s = block_sum(s, red);
  if (threadIdx.x == 0) red[33] = s / (double)N;
  __syncthreads();
  const double mean = red[33];
  __syncthreads();
  double v = 0.0;
  for (int64_t q = threadIdx.x; q < N; q += blockDim.x) {
    const double d = log1p(F[q * kFeat + j]) - mean;
    v += d * d;
  }
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    const double sdv = sqrt(v / (double)N);
    mu[j] = (float)mean;
    sd[j] = sdv > 0.0 ? (float)sdv : 1.f;
  }
}

__global__ void k_feat_standardise(int64_t N, const double* __restrict__ F,
                                   const float* __restrict__ mu, const float* __restrict__ sd,
                                   float* __restrict__ X) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < N * kFeat;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(q % kFeat);
    X[q] = (float)((log1p(F[q]) - (double)mu[j]) / (double)sd[j]);
  }
}

struct Feat15 {
  double f[kFeat];
};

// One block: classify one feature vector; writes the arg-max class (first on
// ties) to *out.
__global__ void k_mlp_infer(Feat15 F, MlpDims D, const float* __restrict__ P,
                            const float* __restrict__ mu, const float* __restrict__ sd,
                            int* __restrict__ out, float* __restrict__ logits) {
  __shared__ float z[kFeat];
  __shared__ float a1[kMaxHidden], a2[kMaxHidden], lg[kMaxClass];
  const float* W1 = P;
  const float* b1 = W1 + D.h1 * D.d;
  const float* W2 = b1 + D.h1;
  const float* b2 = W2 + D.h2 * D.h1;
  const float* W3 = b2 + D.h2;
  const float* b3 = W3 + D.k * D.h2;
  const int t = threadIdx.x;
  if (t < kFeat) z[t] = (float)((log1p(F.f[t]) - (double)mu[t]) / (double)sd[t]);
  __syncthreads();
  if (t < D.h1) {
    float acc = b1[t];
    for (int i = 0; i < D.d; ++i) acc = fmaf(W1[t * D.d + i], z[i], acc);
    a1[t] = acc > 0.f ? acc : 0.f;
  }
  __syncthreads();
  if (t < D.h2) {
    float acc = b2[t];
    for (int i = 0; i < D.h1; ++i) acc = fmaf(W2[t * D.h1 + i], a1[i], acc);
    a2[t] = acc > 0.f ? acc : 0.f;
  }
  __syncthreads();
  if (t < D.k) {
    float acc = b3[t];
    for (int i = 0; i < D.h2; ++i) acc = fmaf(W3[t * D.h2 + i], a2[i], acc);
    lg[t] = acc;
  }
  __syncthreads();
  if (t == 0) {
    int best = 0;
    for (int o = 1; o < D.k; ++o)
      if (lg[o] > lg[best]) best = o;
    *out = best;
    if (logits)
      for (int o = 0; o < D.k; ++o) logits[o] = lg[o];
  }
}

// ------------------------------------------------------------------ host: kernels
static int grid_small(int64_t items) {
  int64_t g = (items + 127) / 128;
  if (g > 1184) g = 1184;
  return (int)(g < 1 ? 1 : g);
}

static void check_dims(const MlpDims& D) {
  CP_REQUIRE(D.d == kFeat || (D.d >= 1 && D.d <= 64), CP_ERR_INVALID, "bad input width %d", D.d);
  CP_REQUIRE(D.h1 >= 1 && D.h1 <= kMaxHidden && D.h2 >= 1 && D.h2 <= kMaxHidden, CP_ERR_INVALID,
             "hidden widths must be in 1..%d", kMaxHidden);
  CP_REQUIRE(D.k >= 2 && D.k <= kMaxClass, CP_ERR_INVALID, "classes must be in 2..%d", kMaxClass);
}

void mlp_forward(cp_ctx* ctx, int64_t N, MlpDims D, const float* P, const float* X, float* Z,
                 float* scratch, cudaStream_t s) {
  check_dims(D);
  float* A1 = scratch;
  float* A2 = A1 + N * D.h1;
  CP_LAUNCH(ctx, k_mlp_fwd, grid_small(N), 128, 0, s, N, D, P, X, A1, A2, Z);
}

void mlp_loss_grad(cp_ctx* ctx, int64_t N, MlpDims D, const float* P, const float* X,
                   const int32_t* lab, const float* Q, float* loss, float* grad, float* scratch,
                   cudaStream_t s) {
  check_dims(D);
  float* A1 = scratch;
  float* A2 = A1 + N * D.h1;
  float* Z = A2 + N * D.h2;
  float* G1 = Z + N * D.k;
  float* G2 = G1 + N * D.h1;
  float* G3 = G2 + N * D.h2;
  float* L = G3 + N * D.k;
  CP_LAUNCH(ctx, k_mlp_fwd, grid_small(N), 128, 0, s, N, D, P, X, A1, A2, Z);
  CP_LAUNCH(ctx, k_mlp_bwd, grid_small(N), 128, 0, s, N, D, P, lab, Q, A1, A2, Z, G1, G2, G3, L);
  CP_LAUNCH(ctx, k_mlp_grad, grid_small(D.nparams()), 128, 0, s, N, D, X, A1, A2, G1, G2, G3,
            grad);
  CP_LAUNCH(ctx, k_mlp_loss, 1, 256, 0, s, N, L, loss);
}

void adam_step(cp_ctx* ctx, int64_t np, float* P, const float* G, float* m, float* v, int t,
               float lr, float b1, float b2, float eps, cudaStream_t s) {
  CP_REQUIRE(t >= 1, CP_ERR_INVALID, "Adam step count must be >= 1");
  const float c1 = (float)(1.0 - std::pow((double)b1, t));
  const float c2 = (float)(1.0 - std::pow((double)b2, t));
  CP_LAUNCH(ctx, k_adam, grid_small(np), 128, 0, s, np, P, G, m, v, lr, b1, b2, eps, c1, c2);
}

// ------------------------------------------------------------------ host: models
void model_install(cp_ctx* ctx, int stage, int h1, int h2, int k, const float* params_dev,
                   const float* mu_dev, const float* sd_dev, cudaStream_t s, uint64_t gen) {
  CP_REQUIRE(stage >= 0 && stage < CP_NUM_STAGES, CP_ERR_INVALID, "bad stage %d", stage);
  const MlpDims D{kFeat, h1, h2, k};
  check_dims(D);
  static const int expect_k[CP_NUM_STAGES] = {CP_NUM_FMT, CP_NUM_ALGO, 5, 4, 3};
  CP_REQUIRE(k == expect_k[stage], CP_ERR_INVALID, "stage %d needs %d classes, got %d", stage,
             expect_k[stage], k);
  ModelSlot fresh;
  fresh.h1 = h1;
  fresh.h2 = h2;
  fresh.k = k;
  fresh.d_params = dalloc<float>(D.nparams());
  fresh.d_mu = dalloc<float>(kFeat);
  fresh.d_sd = dalloc<float>(kFeat);
  CP_CUDA(cudaMemcpyAsync(fresh.d_params, params_dev, D.nparams() * 4, cudaMemcpyDefault, s));
  CP_CUDA(cudaMemcpyAsync(fresh.d_mu, mu_dev, kFeat * 4, cudaMemcpyDefault, s));
  CP_CUDA(cudaMemcpyAsync(fresh.d_sd, sd_dev, kFeat * 4, cudaMemcpyDefault, s));
  CP_CUDA(cudaStreamSynchronize(s));
  fresh.loaded = true;
  static std::atomic<uint64_t> installs{0};
  fresh.gen = gen ? gen : installs.fetch_add(1) + 1;
  std::lock_guard<std::mutex> lock(ctx->model_mu);
  ModelSlot& old = ctx->models[stage];
  dfree(old.d_params);
  dfree(old.d_mu);
  dfree(old.d_sd);
  old = fresh;
}

int infer_stage(cp_ctx* ctx, int stage, const double* f15, cudaStream_t s, float* logits) {
  ModelSlot slot;
  {
    std::lock_guard<std::mutex> lock(ctx->model_mu);
    slot = ctx->models[stage];
  }
  if (!slot.loaded) return -1;
  Feat15 F;
  std::memcpy(F.f, f15, sizeof(F.f));
  // one staging word for the pick, then the k logits (one copy back)
  int* d_out = nullptr;
  CP_CUDA(cudaMallocAsync(&d_out, sizeof(int) * (1 + kMaxClass), s));
  const MlpDims D{kFeat, slot.h1, slot.h2, slot.k};
  int h_out[1 + kMaxClass] = {-1};
  CP_LAUNCH(ctx, k_mlp_infer, 1, 64, 0, s, F, D, slot.d_params, slot.d_mu, slot.d_sd, d_out,
            reinterpret_cast<float*>(d_out + 1));
  d2h_small(ctx, h_out, d_out, sizeof(int) * (1 + slot.k), s);
  CP_CUDA(cudaFreeAsync(d_out, s));
  if (logits) std::memcpy(logits, h_out + 1, sizeof(float) * slot.k);
  return h_out[0];
}

uint64_t model_generation(cp_ctx* ctx, int stage) {
  std::lock_guard<std::mutex> lock(ctx->model_mu);
  return ctx->models[stage].loaded ? ctx->models[stage].gen : 0;
}

int stage_classes(cp_ctx* ctx, int stage) {
  std::lock_guard<std::mutex> lock(ctx->model_mu);
  return ctx->models[stage].loaded ? ctx->models[stage].k : 0;
}

void model_train(cp_ctx* ctx, int stage, int64_t N, const double* F_host, const int32_t* lab_host,
                 const float* q_host, int h1, int h2, int k, int epochs, float lr, uint64_t seed,
                 float* final_loss) {
  CP_REQUIRE(N >= 1, CP_ERR_INVALID, "no training samples");
  CP_REQUIRE((lab_host != nullptr) != (q_host != nullptr), CP_ERR_INVALID,
             "give either labels or target distributions");
  const MlpDims D{kFeat, h1, h2, k};
  check_dims(D);
  if (lab_host)
    for (int64_t q = 0; q < N; ++q)
      CP_REQUIRE(lab_host[q] >= 0 && lab_host[q] < k, CP_ERR_INVALID, "label %d out of range",
                 lab_host[q]);
  if (q_host)
    for (int64_t q = 0; q < N; ++q) {
      double sum = 0.0;
      for (int o = 0; o < k; ++o) {
        const float v = q_host[q * k + o];
        CP_REQUIRE(v >= 0.f && std::isfinite(v), CP_ERR_INVALID, "target of sample %lld is not a "
                   "distribution", (long long)q);
        sum += v;
      }
      CP_REQUIRE(std::fabs(sum - 1.0) <= 1e-4, CP_ERR_INVALID,
                 "targets of sample %lld sum to %g, not 1", (long long)q, sum);
    }
  cudaStream_t s = ctx->main;
  const int64_t np = D.nparams();
  // Glorot-uniform initial weights from a splitmix64 stream, zero biases
  std::vector<float> P0(np, 0.f);
  uint64_t st = seed;
  auto next = [&st]() {
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
  };
  auto fill = [&](int64_t off, int fo, int fi) {
    const double a = std::sqrt(6.0 / (fo + fi));
    for (int64_t i = 0; i < (int64_t)fo * fi; ++i) P0[off + i] = (float)((2.0 * next() - 1.0) * a);
  };
  fill(0, h1, kFeat);
  fill((int64_t)h1 * kFeat + h1, h2, h1);
  fill((int64_t)h1 * kFeat + h1 + (int64_t)h2 * h1 + h2, k, h2);

  std::vector<void*> bufs;
  auto get = [&](size_t bytes) {
    void* p = nullptr;
    CP_CUDA(cudaMalloc(&p, bytes));
    bufs.push_back(p);
    return p;
  };
  try {
    double* dF = static_cast<double*>(get(N * kFeat * 8));
    int32_t* dL = lab_host ? static_cast<int32_t*>(get(N * 4)) : nullptr;
    float* dQ = q_host ? static_cast<float*>(get(N * k * 4)) : nullptr;
    float* X = static_cast<float*>(get(N * kFeat * 4));
    float* mu = static_cast<float*>(get(kFeat * 4));
    float* sd = static_cast<float*>(get(kFeat * 4));
    float* P = static_cast<float*>(get(np * 4));
    float* G = static_cast<float*>(get(np * 4));
    float* M = static_cast<float*>(get(np * 4));
    float* Vv = static_cast<float*>(get(np * 4));
    float* loss = static_cast<float*>(get(4));
    float* scratch = static_cast<float*>(get(scratch_floats(N, D) * 4));
    CP_CUDA(cudaMemcpyAsync(dF, F_host, N * kFeat * 8, cudaMemcpyHostToDevice, s));
    if (dL) CP_CUDA(cudaMemcpyAsync(dL, lab_host, N * 4, cudaMemcpyHostToDevice, s));
    if (dQ) CP_CUDA(cudaMemcpyAsync(dQ, q_host, N * k * 4, cudaMemcpyHostToDevice, s));
    CP_CUDA(cudaMemcpyAsync(P, P0.data(), np * 4, cudaMemcpyHostToDevice, s));
    CP_CUDA(cudaMemsetAsync(M, 0, np * 4, s));
    CP_CUDA(cudaMemsetAsync(Vv, 0, np * 4, s));
    CP_LAUNCH(ctx, k_feat_stats, kFeat, 256, 0, s, N, dF, mu, sd);
    CP_LAUNCH(ctx, k_feat_standardise, grid_small(N * kFeat), 128, 0, s, N, dF, mu, sd, X);
    for (int t = 1; t <= epochs; ++t) {
      mlp_loss_grad(ctx, N, D, P, X, dL, dQ, loss, G, scratch, s);
      adam_step(ctx, np, P, G, M, Vv, t, lr, 0.9f, 0.999f, 1e-8f, s);
    }
    mlp_loss_grad(ctx, N, D, P, X, dL, dQ, loss, G, scratch, s);
    float h_loss = 0.f;
    CP_CUDA(cudaMemcpyAsync(&h_loss, loss, 4, cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaStreamSynchronize(s));
    if (final_loss) *final_loss = h_loss;
    model_install(ctx, stage, h1, h2, k, P, mu, sd, s);
  } catch (...) {
    for (void* p : bufs) cudaFree(p);
    throw;
  }
  for (void* p : bufs) cudaFree(p);
}

// ------------------------------------------------------------------ the cascade
static const int kTpvClasses[5] = {2, 4, 8, 16, 32};
static const int kSigmaClasses[4] = {1, 32, 1024, 8192};

// Threads per row when a CSR-vector kernel is chosen without a TpV model:
// the power of two nearest the mean row length, clamped to [2, 32].
static int tpv_heuristic(const double* f) {
  int t = 2;
  while (t < 32 && t < f[4]) t <<= 1;
  return t;
}

double gate_knn_speedup(int count, int k, const double* mu, const double* sd, const float* z,
                        const float* speedup, const double* features, int fmt) {
  if (k > count) k = count;
  double q[kFeat];
  for (int i = 0; i < kFeat; ++i) q[i] = (std::log1p(std::max(features[i], 0.0)) - mu[i]) / sd[i];
  // squared distances, then the k smallest (ties to the lower index)
  std::vector<std::pair<double, int>> d(count);
  for (int j = 0; j < count; ++j) {
    double s2 = 0.0;
    for (int i = 0; i < kFeat; ++i) {
      const double t = (double)z[(int64_t)j * kFeat + i] - q[i];
      s2 += t * t;
    }
    d[j] = {s2, j};
  }
  std::partial_sort(d.begin(), d.begin() + k, d.end());
  std::vector<double> v(k);
  for (int j = 0; j < k; ++j) v[j] = speedup[(int64_t)d[j].second * CP_NUM_FMT + fmt];
  std::sort(v.begin(), v.end());
  return (k & 1) ? v[k / 2] : 0.5 * (v[k / 2 - 1] + v[k / 2]);
}

// The rule's two figures for format fmt (fmt < 0: the first tier's best
// case): the conversion's cost in default-kernel SpMVs (kappa) and the SpMV
// speedup (s).
static void gate_terms(const cp_gate& g, int fmt, int64_t nnz, double* kappa, double* speedup) {
  const double mnnz = (double)nnz * 1e-6;
  const double t_spmv = g.spmv_a_ms + g.spmv_b_ms * mnnz;
  double t_conv, s;
  if (fmt > 0) {
    t_conv = g.conv_a_ms[fmt] + g.conv_b_ms[fmt] * mnnz;
    s = g.speedup[fmt];
  } else {  // first tier: the best case over the formats, features included
    t_conv = 1e300;
    s = 1.0;
    for (int f = 1; f < CP_NUM_FMT; ++f) {
      t_conv = std::min(t_conv, g.conv_a_ms[f] + g.conv_b_ms[f] * mnnz);
      s = std::max(s, g.speedup[f]);
    }
    t_conv += g.feat_a_ms + g.feat_b_ms * mnnz;
  }
  *kappa = t_spmv > 0.0 ? t_conv / t_spmv : 1e300;
  *speedup = s;
}

double gate_payback(const cp_gate& g, int fmt, int64_t nnz) {
  if (!g.enabled || fmt >= CP_NUM_FMT || fmt == 0) return 0.0;  // the rule does not apply
  double kappa, s;
  gate_terms(g, fmt, nnz, &kappa, &s);
  return s > 1.0 ? kappa / (1.0 - 1.0 / s) : HUGE_VAL;
}

int gate_decide(const cp_gate& g, int fmt, int64_t nnz, int iters, double res0, double res,
                double target, double* remaining, double* cost) {
  double rem = -1.0, kappa = -1.0;
  int go = 1;
  if (g.enabled && fmt < CP_NUM_FMT && fmt != 0) {
    double s;
    gate_terms(g, fmt, nnz, &kappa, &s);
    if (!(s > 1.0)) {
      go = 0;  // no gain expected from the format
    } else if (iters >= 2 && res0 > 0.0 && res > 0.0 && target > 0.0) {
      if (res <= target) {
        rem = 0.0;
        go = 0;
      } else {
        const double rate = std::log(res / res0) / iters;  // < 0 while the residual decays
        if (rate < 0.0) {
          rem = std::log(target / res) / rate;
          go = rem * (1.0 - 1.0 / s) > kappa ? 1 : 0;
        }  // no decay yet: a long solve ahead, switch
      }
    }
  }
  if (remaining) *remaining = rem;
  if (cost) *cost = kappa;
  return go;
}

constexpr int kGateWindow = 8;  // first window over which a "keep" verdict is re-examined
constexpr int kGateRounds = 6;  // windows at most (8, 16, ... iterations)
constexpr double kGateQuick = 4.0;          // payback (iterations) that needs no history
constexpr double kGateQuickMargin = 1e3;    // residual over its target for the quick go

// The solve's progress as its GPU has written it: iterations done (-1: not
// started), latest and initial residual norm, ||b||.
struct Progress {
  int iters = -1;
  double res = 0.0, res0 = 0.0, bnorm = 0.0;
};
static Progress progress(const Channel* ch) {
  Progress p;
  const Mirror* mir = ch->live.load(std::memory_order_acquire);
  if (!mir) return p;
  p.res0 = mir->res0;
  p.bnorm = mir->bnorm;
  p.res = mir->res;
  p.iters = p.res0 > 0.0 ? mir->iters : -1;  // res0 is written when the solve starts
  return p;
}

// Waits (bounded) until the solve has done at least `iters` iterations,
// finished, or the side work was cancelled.
static void wait_progress(Channel* ch, int iters, double max_ms) {
  const auto t0 = std::chrono::steady_clock::now();
  while (progress(ch).iters < iters && !ch->solve_done.load(std::memory_order_acquire) &&
         !ch->cancel.load()) {
    if (std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() >
        max_ms)
      return;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

// The gate: decides on the decay since the start; a "keep" is re-examined on
// later windows (the solve stays on the default kernel meanwhile).  Returns
// true to go on; records the estimates in ch; sets ch->gate_declined to `tier`
// while keeping.
static bool gate_pass(cp_ctx* ctx, cp_mat* m, Channel* ch, int fmt, int tier) {
  double rem = -1.0, cost = -1.0;
  // with the features known and neighbours installed, format fmt's speedup for
  // this matrix: the median over the nearest training matrices
  cp_gate g = ctx->gate;
  if (fmt > 0 && m->has_features) {
    std::lock_guard<std::mutex> lock(ctx->gate_mu);
    const auto& nb = ctx->gate_nb;
    if (nb.count > 0) {
      g.speedup[fmt] = gate_knn_speedup(nb.count, nb.k, nb.mu, nb.sd, nb.z.data(),
                                        nb.speedup.data(), m->features, fmt);
      trace("cascade: gate speedup of format %d from %d neighbours: %.3f", fmt, nb.k,
            g.speedup[fmt]);
    }
  }
  // A switch that pays for itself within kGateQuick default iterations is
  // taken without waiting for history: a solve to the tolerance asked for
  // that ends sooner than that (residual still above kGateQuickMargin x its
  // target) is rare, and a wrong "go" then costs at most about the conversion.
  const double payback = gate_payback(g, fmt, m->nnz);
  {
    const Progress p0 = progress(ch);
    const double target0 = ch->tol * p0.bnorm;
    if (payback <= kGateQuick && (p0.iters < 0 || p0.res > kGateQuickMargin * target0)) {
      gate_decide(g, fmt, m->nnz, 0, 0.0, 0.0, 0.0, &rem, &cost);
      ch->gate_remaining = (float)rem;
      ch->gate_cost = (float)cost;
      trace("cascade: gate (tier %d, format %d): pays back within %.1f iterations -> go", tier,
            fmt, payback);
      return true;
    }
  }
  wait_progress(ch, 2, 5.0);  // two iterations of history (the GPU's own count)
  if (ch->cancel.load()) return false;
  const Progress p = progress(ch);
  const double target = ch->tol * p.bnorm;
  int go = gate_decide(g, fmt, m->nnz, p.iters, p.res0, p.res, target, &rem, &cost);
  ch->gate_remaining = (float)rem;
  ch->gate_cost = (float)cost;
  trace("cascade: gate (tier %d, format %d): %d iterations left, cost %.1f SpMVs -> %s", tier,
        fmt, (int)rem, cost, go ? "go" : "keep (to be confirmed)");
  if (go) return true;
  // Krylov residuals often drop fast in the first iterations and slow down
  // later, so a "keep" is re-examined on later windows of doubling length
  // while the estimate of the iterations left keeps growing (by more than a
  // quarter per window); a steady estimate makes it final
  ch->gate_declined = tier;
  // only host waits follow until the verdict: the solve may use the whole GPU
  // (the persistent kernel), and is asked to return if the verdict turns to go
  struct Idle {
    Channel* c;
    explicit Idle(Channel* ch) : c(ch) { c->side_gpu_idle.store(true, std::memory_order_release); }
    ~Idle() { c->side_gpu_idle.store(false, std::memory_order_release); }
  } idle(ch);
  int k1 = p.iters;
  double r1 = p.res, est = rem;
  int w = std::max(kGateWindow, k1);
  for (int round = 0; round < kGateRounds; ++round, w *= 2) {
    wait_progress(ch, k1 + w, 50.0);
    if (ch->cancel.load()) return false;
    const Progress q = progress(ch);
    if (q.iters <= k1) return false;
    go = gate_decide(g, fmt, m->nnz, q.iters - k1, r1, q.res, target, &rem, &cost);
    ch->gate_remaining = (float)rem;
    ch->gate_cost = (float)cost;
    trace("cascade: gate window %d..%d: %d iterations left -> %s", k1, q.iters, (int)rem,
          go ? "go" : "keep");
    if (go) {
      ch->gate_declined = 0;
      return true;
    }
    if (!(rem > 1.25 * est)) return false;  // the estimate has settled
    est = rem;
    k1 = q.iters;
    r1 = q.res;
  }
  return false;
}

// Host fault injection (cp_inject_side_failure): one-shot, at `point`.
static void maybe_fail(cp_ctx* ctx, int point) {
  int want = point;
  if (ctx->inject_side_fail.compare_exchange_strong(want, -1))
    throw Error{CP_ERR_CUDA};  // as a failing CUDA call would
}

void run_cascade(cp_ctx* ctx, cp_mat* m, cudaStream_t s, Channel* ch) {
  struct Finish {  // tell the solve loop the side work has ended, however it ends
    Channel* c;
    ~Finish() { c->finished.store(true, std::memory_order_release); }
  } finish{ch};
  using Clock = std::chrono::steady_clock;
  auto ms = [](Clock::time_point a) {
    return (float)std::chrono::duration<double, std::milli>(Clock::now() - a).count();
  };
  try {
    CP_CUDA(cudaSetDevice(ctx->device));  // the side thread's CUDA calls target ctx's GPU
    trace("cascade: side thread started");
    if (ctx->gate.enabled && ch->tol > 0.0 && m->nrows < ctx->gate.small_rows) {
      // two-tier features: on a small matrix the O(nnz) feature pass is run
      // only if the best case over the formats can pay for it
      if (!gate_pass(ctx, m, ch, -1, 2)) return;
    }
    maybe_fail(ctx, 0);
    auto t = Clock::now();
    double f[kFeat];
    compute_features(ctx, m, s, f);  // Table IV, on the side stream
    ch->t_features_ms = ms(t);
    if (ch->cancel.load()) return;
    maybe_fail(ctx, 1);

    cp_config cfg;
    cp_config_default(&cfg);
    // stage 1: FORMAT (with SELL's sort window, which its conversion needs)
    t = Clock::now();
    int fmt = infer_stage(ctx, CP_STAGE_FORMAT, f, s);
    cp_config next = cfg;
    if (fmt > 0) {
      next.fmt = fmt;
      if (fmt == CP_FMT_SELL) {
        const int sg = infer_stage(ctx, CP_STAGE_SELL_SIGMA, f, s);
        next.sell_sigma = kSigmaClasses[sg >= 0 ? sg : 2];
      }
    }
    ch->t_predict_ms[0] = ms(t);
    trace("cascade: FORMAT -> %d", next.fmt);
    if (ch->cancel.load()) return;
    maybe_fail(ctx, 2);
    if (next.fmt != cfg.fmt && ctx->gate.enabled && ch->tol > 0.0) {
      // cost-aware switching: convert only if the saving over the iterations
      // left pays for the conversion.  The gate waits at most 5 ms for two
      // iterations of history; without it the solve counts as long.
      if (!gate_pass(ctx, m, ch, next.fmt, 1)) return;
    }
    if (next.fmt != cfg.fmt) {
      t = Clock::now();
      try {
        ensure_format(ctx, m, next, s);
        if (ch->need_fp32) ensure_val32(ctx, m, next, s);
        cfg = next;
      } catch (const Error& e) {
        // a padded format over budget: stay on CSR (the plain fallback)
        if (e.status != CP_ERR_FOOTPRINT) throw;
      }
      ch->t_convert_ms = ms(t);
      trace("cascade: converted, publishing format %d", cfg.fmt);
      if (cfg.fmt != CP_FMT_CSR) ch->publish(0, cfg);
    }
    if (ch->cancel.load() || cfg.fmt != CP_FMT_CSR) return;
    // stage 2: the CSR algorithm
    t = Clock::now();
    const int algo = infer_stage(ctx, CP_STAGE_CSR_ALGO, f, s);
    ch->t_predict_ms[1] = ms(t);
    if (algo > 0) {
      cfg.algo = algo;
      if (algo == CP_ALGO_VECTOR) cfg.tpv = tpv_heuristic(f);
      ensure_format(ctx, m, cfg, s);
      ch->publish(1, cfg);
    }
    if (ch->cancel.load() || cfg.algo != CP_ALGO_VECTOR) return;
    // stage 3: threads per row of the CSR-vector kernel
    t = Clock::now();
    const int tp = infer_stage(ctx, CP_STAGE_CSR_TPV, f, s);
    ch->t_predict_ms[2] = ms(t);
    if (tp >= 0 && kTpvClasses[tp] != cfg.tpv) {
      cfg.tpv = kTpvClasses[tp];
      ch->publish(2, cfg);
    }
  } catch (const Error& e) {
    ch->status = e.status;
    ch->error = "prediction failed";
  } catch (...) {
    ch->status = CP_ERR_CUDA;
    ch->error = "prediction failed";
  }
}

int64_t scratch_floats_api(int64_t N, int d, int h1, int h2, int k) {
  return scratch_floats(N, MlpDims{d, h1, h2, k});
}

}  // namespace cp
