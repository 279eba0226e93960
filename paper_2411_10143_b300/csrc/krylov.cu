// Krylov solvers around the SpMV family: CG (Hestenes-Stiefel) and restarted
// GMRES(m), in FP64 or as FP32 inner solves inside FP64 iterative refinement,
// with the paper's asynchronous execution (Sec. III-C-2): the solve starts at
// once on the default kernel while the side thread extracts features, runs the
// cascade and converts the format on the side stream; the loop adopts each
// published configuration at the next iteration boundary (Table VII records
// where), and cancels the side work if it converges first.
//
// Scalars (alpha, beta, residual norms, Givens rotations) live in device
// memory and every reduction is a fixed-order sum of per-block partials, so the
// host never waits on the GPU inside an iteration: it runs at most
// check_every iterations ahead and reads a host-mapped mirror of the state.
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.cuh"
#include "gm_state.cuh"
#include "persist.cuh"
#include "spmv_rows.cuh"

namespace cp {

// ================================================================== CG kernels
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_init(int64_t n, const T* __restrict__ b,
                                                    const T* __restrict__ ax, T* __restrict__ r,
                                                    T* __restrict__ p, double* __restrict__ pr,
                                                    double* __restrict__ pb) {
  T rr = 0, bb = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T bi = b[i];
    const T ri = ax ? bi - ax[i] : bi;
    r[i] = ri;
    p[i] = ri;
    rr = fma(ri, ri, rr);
    bb = fma(bi, bi, bb);
  }
  __shared__ double red[33];
  const double s1 = block_sum((double)rr, red);
  if (threadIdx.x == 0) pr[blockIdx.x] = s1;
  const double s2 = block_sum((double)bb, red);
  if (threadIdx.x == 0) pb[blockIdx.x] = s2;
}

// One block: (r, r) and ||b||^2 into the state; converged already?
__global__ void k_cg_init_final(const double* __restrict__ pr, const double* __restrict__ pb,
                                int P, CgState* st, int slot, double tol2, Mirror* mir,
                                int keep_bb) {
  __shared__ double red[40];
  const double rr = reduce_partials(pr, P, red);
  const double bb = keep_bb ? st->bb : reduce_partials(pb, P, red);
  if (threadIdx.x == 0) {
    st->rr[slot] = rr;
    st->bb = bb;
    const int done = (bb == 0.0 || rr <= tol2 * bb) ? 1 : 0;
    st->done = done;
    st->status = CP_OK;
    mir->res = sqrt(rr);
    mir->res0 = sqrt(rr);
    mir->bnorm = sqrt(bb);
    mir->done = done;
    mir->status = CP_OK;
    mir->iters = st->iters;
  }
}

// The two CG vector kernels move pairs of values (16-byte FP64 / 8-byte FP32
// loads) in tiles of kBlock * kVecU pairs per block.  Each block issues the
// loads of its first tile before it sums the previous kernel's partials, so
// the reduction's latency hides behind the DRAM latency.  An odd last element
// is handled by block 0.
constexpr int kVecU = 2;

// alpha = (r,r)/(Ap,p); x += alpha p; r -= alpha Ap; partials of (r,r).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_update(int64_t n, T* __restrict__ x,
                                                      T* __restrict__ r, const T* __restrict__ p,
                                                      const T* __restrict__ ap,
                                                      const double* __restrict__ pa, int PA,
                                                      CgState* st, int slot,
                                                      double* __restrict__ pb, Mirror* mir) {
  if (*(volatile int*)&st->done) return;
  using V = typename Vec2<T>::type;
  V* __restrict__ x2 = reinterpret_cast<V*>(x);
  V* __restrict__ r2 = reinterpret_cast<V*>(r);
  const V* __restrict__ p2 = reinterpret_cast<const V*>(p);
  const V* __restrict__ a2 = reinterpret_cast<const V*>(ap);
  const int64_t n2 = n >> 1;
  const int64_t tile = (int64_t)blockDim.x * kVecU;
  const int64_t ntiles = (n2 + tile - 1) / tile;
  V xv[kVecU], rv[kVecU], pv[kVecU], av[kVecU];
  int64_t t = blockIdx.x;
  auto load = [&](int64_t tt) {
#pragma unroll
    for (int u = 0; u < kVecU; ++u) {
      const int64_t idx = tt * tile + (int64_t)u * blockDim.x + threadIdx.x;
      if (idx < n2) {
        xv[u] = x2[idx];
        rv[u] = r2[idx];
        pv[u] = p2[idx];
        av[u] = a2[idx];
      }
    }
  };
  if (t < ntiles) load(t);
  __shared__ double red[40];
  __shared__ double sc_alpha;
  __shared__ int sc_bad;
  const double pap = partials_sum0(pa, PA, red);
  if (threadIdx.x == 0) {  // alpha formed once per block
    const bool bad = !(pap > 0.0) || !isfinite(pap);  // A not SPD, or overflow / NaN
    const double alpha_d = bad ? 0.0 : st->rr[slot] / pap;
    sc_alpha = alpha_d;
    sc_bad = bad;
    if (blockIdx.x == 0) {
      if (bad) {
        st->status = CP_ERR_BREAKDOWN;
        st->done = 1;
        mir->status = CP_ERR_BREAKDOWN;
        mir->done = 1;
      } else {
        st->pap = pap;
        st->alpha = alpha_d;
      }
    }
  }
  __syncthreads();
  if (sc_bad) return;
  const T alpha = (T)sc_alpha;
  T acc = 0;
  for (; t < ntiles; t += gridDim.x) {
    if (t != blockIdx.x) load(t);
#pragma unroll
    for (int u = 0; u < kVecU; ++u) {
      const int64_t idx = t * tile + (int64_t)u * blockDim.x + threadIdx.x;
      if (idx < n2) {
        V xn, rn;
        xn.x = fma(alpha, pv[u].x, xv[u].x);
        xn.y = fma(alpha, pv[u].y, xv[u].y);
        rn.x = fma(-alpha, av[u].x, rv[u].x);
        rn.y = fma(-alpha, av[u].y, rv[u].y);
        x2[idx] = xn;
        r2[idx] = rn;
        acc = fma(rn.x, rn.x, acc);
        acc = fma(rn.y, rn.y, acc);
      }
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    const int64_t i = n - 1;
    x[i] = fma(alpha, p[i], x[i]);
    const T ri = fma(-alpha, ap[i], r[i]);
    r[i] = ri;
    acc = fma(ri, ri, acc);
  }
  const double s = block_sum((double)acc, red);
  if (threadIdx.x == 0) pb[blockIdx.x] = s;
}

// beta = (r+,r+)/(r,r); p = r + beta p, unless converged.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_cg_direction(int64_t n, const T* __restrict__ r,
                                                         T* __restrict__ p,
                                                         const double* __restrict__ pb, int PB,
                                                         CgState* st, int slot, double tol2,
                                                         Mirror* mir) {
  if (*(volatile int*)&st->done) return;
  using V = typename Vec2<T>::type;
  const V* __restrict__ r2 = reinterpret_cast<const V*>(r);
  V* __restrict__ p2 = reinterpret_cast<V*>(p);
  const int64_t n2 = n >> 1;
  const int64_t tile = (int64_t)blockDim.x * kVecU * 2;
  const int64_t ntiles = (n2 + tile - 1) / tile;
  constexpr int U = kVecU * 2;
  V rv[U], pv[U];
  int64_t t = blockIdx.x;
  auto load = [&](int64_t tt) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t idx = tt * tile + (int64_t)u * blockDim.x + threadIdx.x;
      if (idx < n2) {
        rv[u] = r2[idx];
        pv[u] = p2[idx];
      }
    }
  };
  if (t < ntiles) load(t);
  __shared__ double red[40];
  __shared__ double sc_beta;
  __shared__ int sc_stop;
  const double rr_new = partials_sum0(pb, PB, red);
  if (threadIdx.x == 0) {  // beta and the stopping test, once per block
    const bool bad = !isfinite(rr_new);
    const bool conv = rr_new <= tol2 * st->bb;
    const double beta_d = rr_new / st->rr[slot];
    sc_beta = beta_d;
    sc_stop = conv || bad;
    if (blockIdx.x == 0) {
      st->rr[slot ^ 1] = rr_new;
      st->iters += 1;
      mir->res = sqrt(rr_new);
      mir->iters = st->iters;
      if (bad) {
        st->status = CP_ERR_BREAKDOWN;
        mir->status = CP_ERR_BREAKDOWN;
      }
      if (conv || bad) {
        st->done = 1;
        mir->done = 1;
      } else {
        st->beta = beta_d;
      }
    }
  }
  __syncthreads();
  if (sc_stop) return;
  const T beta = (T)sc_beta;
  for (; t < ntiles; t += gridDim.x) {
    if (t != blockIdx.x) load(t);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t idx = t * tile + (int64_t)u * blockDim.x + threadIdx.x;
      if (idx < n2) {
        V pn;
        pn.x = fma(beta, pv[u].x, rv[u].x);
        pn.y = fma(beta, pv[u].y, rv[u].y);
        p2[idx] = pn;
      }
    }
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) p[n - 1] = fma(beta, p[n - 1], r[n - 1]);
}

// ================================================================== shared small kernels
// partials of ||b - y||^2 and, if out is non-null, out = b - y
template <typename T>
__global__ void __launch_bounds__(kBlock) k_resid(int64_t n, const T* __restrict__ b,
                                                  const T* __restrict__ y, T* __restrict__ out,
                                                  double* __restrict__ part, const int* skip) {
  if (skip && *skip) return;
  T acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T d = b[i] - y[i];
    if (out) out[i] = d;
    acc = fma(d, d, acc);
  }
  __shared__ double red[33];
  const double s = block_sum((double)acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_to(const double* __restrict__ part, int P, double* out) {
  __shared__ double red[40];
  const double s = reduce_partials(part, P, red);
  if (threadIdx.x == 0) *out = s;
}

template <typename A, typename B>
__global__ void k_cast(int64_t n, const A* __restrict__ a, B* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (B)a[i];
}
template <>
__global__ void k_cast<double, float>(int64_t n, const double* __restrict__ a,
                                      float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __double2float_rn(a[i]);
}

// x += (double) d
__global__ void k_add_f32(int64_t n, double* __restrict__ x, const float* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

// ================================================================== GMRES kernels
// Multi-dot of w with columns V[c0 .. c0+R) (and, with NORM, (w, w) as one
// more column): partials[(c0 + g) * P + block].  R is exact (no padding
// columns: an idle FMA slot costs the FP64 pipe as much as a used one).
template <typename T, int R, bool NORM>
__device__ __forceinline__ void gm_dots_group(int64_t n, const T* __restrict__ V, int64_t ldv,
                                              int c0, int nc, const T* __restrict__ w,
                                              double* __restrict__ part, double* red) {
  constexpr int G = R + (NORM ? 1 : 0);
  T acc[G];
#pragma unroll
  for (int g = 0; g < G; ++g) acc[g] = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T wi = w[i];
    T v[R];
#pragma unroll
    for (int g = 0; g < R; ++g) v[g] = V[(int64_t)(c0 + g) * ldv + i];
#pragma unroll
    for (int g = 0; g < R; ++g) acc[g] = fma(v[g], wi, acc[g]);
    if (NORM) acc[R] = fma(wi, wi, acc[R]);
  }
  double accd[G];
#pragma unroll
  for (int g = 0; g < G; ++g) accd[g] = (double)acc[g];
  block_sum_multi_lean<G>(accd, red);
  if (threadIdx.x == 0) {
    const int P = gridDim.x;
#pragma unroll
    for (int g = 0; g < R; ++g) part[(int64_t)(c0 + g) * P + blockIdx.x] = accd[g];
    if (NORM) part[(int64_t)nc * P + blockIdx.x] = accd[R];
  }
  __syncthreads();
}

constexpr int kGmGroup = 4;  // columns a thread accumulates at once

template <typename T, bool NORM>
__device__ __forceinline__ void gm_dots_rest(int r, int64_t n, const T* V, int64_t ldv, int c0,
                                             int nc, const T* w, double* part, double* red) {
  switch (r) {
    case 1: gm_dots_group<T, 1, NORM>(n, V, ldv, c0, nc, w, part, red); break;
    case 2: gm_dots_group<T, 2, NORM>(n, V, ldv, c0, nc, w, part, red); break;
    case 3: gm_dots_group<T, 3, NORM>(n, V, ldv, c0, nc, w, part, red); break;
    default: gm_dots_group<T, kGmGroup, NORM>(n, V, ldv, c0, nc, w, part, red); break;
  }
}

// Multi-dot of w with columns V[0..nc): partials[c * P + block], columns in
// groups of kGmGroup (that many accumulators a thread, registers for four
// resident blocks an SM) with an exact last group; the first pass (with_norm)
// also gives (w, w) in column nc.  The second pass returns at once when the
// first left w orthogonal enough (skip2).
template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_gm_dots(int64_t n, const T* __restrict__ V,
                                                       int64_t ldv, int nc,
                                                       const T* __restrict__ w,
                                                       double* __restrict__ part, GmState* st,
                                                       int with_norm) {
  if (*(volatile int*)&st->halt) return;
  if (!with_norm && *(volatile int*)&st->skip2) return;
  __shared__ double red[(kGmGroup + 1) * kBlock + kGmGroup + 1];
  for (int c0 = 0; c0 < nc; c0 += kGmGroup) {
    const int r = nc - c0 < kGmGroup ? nc - c0 : kGmGroup;
    if (with_norm && c0 == 0) gm_dots_rest<T, true>(r, n, V, ldv, c0, nc, w, part, red);
    else gm_dots_rest<T, false>(r, n, V, ldv, c0, nc, w, part, red);
  }
}

// nc blocks: out[c] = sum of column c's partials (fixed order)
__global__ void k_gm_reduce(const double* __restrict__ part, int P, double* out, GmState* st,
                            int pass2) {
  if (*(volatile int*)&st->halt) return;
  if (pass2 && *(volatile int*)&st->skip2) return;
  __shared__ double red[40];
  const double s = reduce_partials(part + (int64_t)blockIdx.x * P, P, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w -= V[:, 0..nc) h; partials of ||w||^2.  The columns go four at a time with
// their loads issued together (an exact last chunk).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gm_sub(int64_t n, const T* __restrict__ V,
                                                   int64_t ldv, int nc, T* __restrict__ w,
                                                   const double* __restrict__ h,
                                                   double* __restrict__ part, GmState* st,
                                                   int pass2) {
  if (*(volatile int*)&st->halt) return;
  if (pass2 && *(volatile int*)&st->skip2) return;
  __shared__ T hs[kMaxRestart + 1];
  for (int c = threadIdx.x; c < nc; c += blockDim.x) hs[c] = (T)h[c];
  __syncthreads();
  T acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T wi = w[i];
    for_slots(nc, [&](int64_t c0, auto R) {
      constexpr int r = decltype(R)::value;
      T v[r];
#pragma unroll
      for (int u = 0; u < r; ++u) v[u] = V[(c0 + u) * ldv + i];
#pragma unroll
      for (int u = 0; u < r; ++u) wi = fma(-hs[c0 + u], v[u], wi);
      return false;
    });
    w[i] = wi;
    acc = fma(wi, wi, acc);
  }
  __shared__ double red[kBlock + 4];
  const double s = block_sum_lean((double)acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// One thread after the first Gram-Schmidt pass: the second pass is needed only
// if the first removed most of w, ||w'|| < ||w|| / sqrt(2) (the criterion of
// Daniel, Gragg, Kaufman and Stewart, 1976); otherwise its coefficients are 0.
// (w, w) before the pass is h1[nc]; ||w'||^2 comes from the partials.
// FP32 solves (the inner solves of the refinement) always take the second
// pass: single precision loses orthogonality too fast for the test to pay.
__global__ void k_gm_reorth_test(const double* __restrict__ part, int P, GmState* st, int nc,
                                 int always) {
  if (*(volatile int*)&st->halt) return;
  __shared__ double red[40];
  const double w2 = reduce_partials(part, P, red);
  if (threadIdx.x != 0) return;
  const double ww = st->h1[nc];
  const int skip = (!always && w2 >= 0.5 * ww) ? 1 : 0;
  st->skip2 = skip;
  if (skip) {
    for (int c = 0; c < nc; ++c) st->h2[c] = 0.0;
  } else {
    st->reorths += 1;
  }
}

// One thread: column j of H from h1 + h2 and ||w||, previous rotations, the new
// rotation, the residual estimate; decides whether the cycle goes on.
__global__ void k_gm_givens(const double* __restrict__ part, int P, GmState* st, int j, int m,
                            double tol2, Mirror* mir) {
  if (*(volatile int*)&st->halt) return;
  __shared__ double red[40];
  const double hn2 = reduce_partials(part, P, red);
  if (threadIdx.x != 0) return;
  const double hn = sqrt(hn2);
  double* H = st->H;
  for (int i = 0; i <= j; ++i) H[i * kMaxRestart + j] = st->h1[i] + st->h2[i];
  for (int i = 0; i < j; ++i) {
    const double a = H[i * kMaxRestart + j], b = H[(i + 1) * kMaxRestart + j];
    H[i * kMaxRestart + j] = st->cs[i] * a + st->sn[i] * b;
    H[(i + 1) * kMaxRestart + j] = -st->sn[i] * a + st->cs[i] * b;
  }
  const double a = H[j * kMaxRestart + j];
  const double den = sqrt(a * a + hn2);
  const double c = den == 0.0 ? 1.0 : a / den;
  const double s = den == 0.0 ? 0.0 : hn / den;
  st->cs[j] = c;
  st->sn[j] = s;
  H[j * kMaxRestart + j] = c * a + s * hn;
  st->g[j + 1] = -s * st->g[j];
  st->g[j] = c * st->g[j];
  st->jdone = j + 1;
  st->iters += 1;
  const double est2 = st->g[j + 1] * st->g[j + 1];
  const bool bad = !isfinite(est2) || !isfinite(hn);
  const bool conv = est2 <= tol2 * st->bb;
  st->conv_est = conv ? 1 : 0;
  st->inv = hn > 0.0 ? 1.0 / hn : 0.0;
  if (bad) st->status = CP_ERR_BREAKDOWN;
  if (conv || hn == 0.0 || bad || j + 1 == m) st->halt = 1;
  mir->res = fabs(st->g[j + 1]);
  mir->iters = st->iters;
  mir->jdone = st->jdone;
  mir->halt = st->halt;
  mir->conv_est = st->conv_est;
  mir->status = st->status;
}

// w *= inv (normalisation of the new basis vector); runs unless halted.
template <typename T>
__global__ void k_gm_scale(int64_t n, T* __restrict__ w, GmState* st, int check_halt) {
  if (check_halt && *(volatile int*)&st->halt) return;
  if (*(volatile int*)&st->done) return;
  const T inv = (T)st->inv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] *= inv;
}

// One thread: cycle start from ||r0||^2 partials (r0 = b - A x already in V0).
__global__ void k_gm_start(const double* __restrict__ part, int P, GmState* st, double tol2,
                           Mirror* mir, int first) {
  if (*(volatile int*)&st->done) return;
  __shared__ double red[40];
  const double rr = reduce_partials(part, P, red);
  if (threadIdx.x != 0) return;
  if (first) st->bb = st->h1[0];  // ||b||^2 staged by the host loop in h1[0]
  const double beta = sqrt(rr);
  st->beta = beta;
  st->jdone = 0;
  st->conv_est = 0;
  for (int i = 0; i <= kMaxRestart; ++i) st->g[i] = 0.0;
  for (int i = 0; i < (kMaxRestart + 1) * kMgsGroupMax; ++i) st->G[i] = 0.0;
  st->g[0] = beta;
  st->inv = beta > 0.0 ? 1.0 / beta : 0.0;
  const bool conv = st->bb == 0.0 || rr <= tol2 * st->bb;
  if (!isfinite(rr)) st->status = CP_ERR_BREAKDOWN;
  st->done = (conv || !isfinite(rr)) ? 1 : 0;
  st->halt = st->done;
  mir->res = beta;
  if (first) {
    mir->res0 = beta;
    mir->bnorm = sqrt(st->bb);
  }
  mir->done = st->done;
  mir->halt = st->halt;
  mir->jdone = 0;
  mir->conv_est = 0;
  mir->status = st->status;
  mir->iters = st->iters;
}

// One thread: y = R^{-1} g over the cycle's jdone steps.
__global__ void k_gm_backsub(GmState* st) {
  if (*(volatile int*)&st->done) return;
  const int jd = st->jdone;
  for (int i = jd - 1; i >= 0; --i) {
    double s = st->g[i];
    for (int k = i + 1; k < jd; ++k) s -= st->H[i * kMaxRestart + k] * st->y[k];
    st->y[i] = s / st->H[i * kMaxRestart + i];
  }
}

// x += V[:, 0..jdone) y
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gm_update_x(int64_t n, const T* __restrict__ V,
                                                        int64_t ldv, T* __restrict__ x,
                                                        GmState* st) {
  if (*(volatile int*)&st->done) return;
  __shared__ T ys[kMaxRestart];
  const int jd = st->jdone;
  for (int c = threadIdx.x; c < jd; c += blockDim.x) ys[c] = (T)st->y[c];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T xi = x[i];
    for (int c = 0; c < jd; ++c) xi = fma(ys[c], V[(int64_t)c * ldv + i], xi);
    x[i] = xi;
  }
}

// ================================================================== host side
using Clock = std::chrono::steady_clock;
static double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

// blocks for a pair-tiled vector kernel: one tile of kBlock * U pairs per block,
// capped at the resident capacity (the kernels loop over further tiles)
static int vec_grid(cp_ctx* ctx, int64_t n, int U) {
  const int64_t tile = (int64_t)kBlock * U;
  int64_t g = ((n >> 1) + tile - 1) / tile;
  if (g > ctx->grid_stream) g = ctx->grid_stream;
  return (int)(g < 1 ? 1 : g);
}

static int grid_n(cp_ctx* ctx, int64_t n) {
  int64_t g = (n + kBlock - 1) / kBlock;
  if (g > ctx->grid_stream) g = ctx->grid_stream;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
struct CgBufs {
  T *r = nullptr, *p = nullptr, *ap = nullptr, *xw = nullptr;
  T* apc = nullptr;  // the COO entries' part of A p in the persistent kernel (HYB, COO)
  double *pa = nullptr, *pb = nullptr, *pc = nullptr;
  CgState* st = nullptr;
};
template <typename T>
struct GmBufs {
  T *V = nullptr, *tmp = nullptr;
  T* wc = nullptr;  // the COO entries' part of A v in the persistent kernel (HYB, COO)
  double *part = nullptr, *part2 = nullptr, *pn = nullptr;
  GmState* st = nullptr;
  int mrest = 0;
};

// Device and host-mapped work areas of one solve (buffers are made once and
// reused by every inner solve of an iterative refinement).  Device buffers come
// from the stream-ordered pool on the solve's stream (the context keeps the
// pool's memory, so an allocation is a pool hit) and go back to it in stream
// order; the host-mapped page and the events come from the context's pools.  A
// solve then spends no time in cudaMalloc / cudaFree / cudaHostAlloc, whose
// frees wait for the whole device.
struct Workspace {
  cp_ctx* ctx;
  std::vector<void*> dev;
  Mirror* mir = nullptr;  // host pointer
  Mirror* mir_d = nullptr;
  std::vector<cudaEvent_t> ring;
  CgBufs<double> cg64;
  CgBufs<float> cg32;
  GmBufs<double> gm64;
  GmBufs<float> gm32;
  explicit Workspace(cp_ctx* c) : ctx(c) {}
  template <typename T>
  CgBufs<T>& cgset();
  template <typename T>
  GmBufs<T>& gmset();
  template <typename T>
  CgBufs<T>& cg(int64_t n) {
    CgBufs<T>& B = cgset<T>();
    if (!B.r) {
      B.r = get<T>(n);
      B.p = get<T>(n);
      B.ap = get<T>(n);
      B.xw = get<T>(n);
      B.pa = get<double>(kMaxPartials);
      B.pb = get<double>(kMaxPartials);
      B.pc = get<double>(kMaxPartials);
      B.st = get<CgState>(1);
    }
    return B;
  }
  template <typename T>
  GmBufs<T>& gm(int64_t n, int64_t ldv, int mrest) {
    GmBufs<T>& B = gmset<T>();
    if (!B.V) {
      B.V = get<T>(ldv * (mrest + 1));
      B.tmp = get<T>(n);
      B.part = get<double>((int64_t)kMaxPartials * (kMaxRestart + 2));
      B.part2 = get<double>((int64_t)kMaxPartials * (kMaxRestart + 2));
      B.pn = get<double>(kMaxPartials);
      B.st = get<GmState>(1);
      B.mrest = mrest;
    }
    return B;
  }
  template <typename U>
  U* get(size_t count) {
    U* p = dalloc_async<U>(count, ctx->main);
    dev.push_back(p);
    return p;
  }
  // one host-mapped page: the mirror at its start, the yield flag after it
  void* page = nullptr;
  char* page_d = nullptr;
  static constexpr size_t kYieldOffset = 1024;
  static_assert(sizeof(Mirror) <= kYieldOffset, "mirror overlaps the yield flag");
  void map_page() {
    if (page) return;
    page = ctx->mapped.take();
    CP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&page_d), page, 0));
    mir = static_cast<Mirror*>(page);
    mir_d = reinterpret_cast<Mirror*>(page_d);
    yield_h = reinterpret_cast<int*>(static_cast<char*>(page) + kYieldOffset);
    yield_d = reinterpret_cast<int*>(page_d + kYieldOffset);
  }
  int* yield_h = nullptr;  // host-mapped flag asking the persistent kernel to return
  int* yield_d = nullptr;
  int* yield() {
    map_page();
    return yield_d;
  }
  Mirror* mirror() {
    map_page();
    return mir_d;
  }
  cudaEvent_t event(int i, int depth) {
    while ((int)ring.size() < depth) ring.push_back(ctx->events.take(false));
    return ring[i % depth];
  }
  ~Workspace() {
    for (void* p : dev) dfree_async(p, ctx->main);
    for (auto e : ring) ctx->events.give(e, false);
    if (page) ctx->mapped.give(page);
  }
};

template <>
CgBufs<double>& Workspace::cgset<double>() { return cg64; }
template <>
CgBufs<float>& Workspace::cgset<float>() { return cg32; }
template <>
GmBufs<double>& Workspace::gmset<double>() { return gm64; }
template <>
GmBufs<float>& Workspace::gmset<float>() { return gm32; }

// The configuration in force, fed by the cascade channel.
struct ConfigSource {
  cp_ctx* ctx;
  cp_mat* m;
  cp_config cur;
  Channel* ch = nullptr;  // null: fixed configuration
  int applied = 0;
  int switch_iter[3] = {-1, -1, -1};
  bool fp32 = false;
  // profiling of SpMV launches
  bool profile = false;
  std::vector<cudaEvent_t> ev;
  int n_spmv = 0;
  bool persistent = true;     // run CG iterations in the persistent kernel when it supports cfg
  double wait_limit_ms = 0.0; // bound of the persistent kernel's device waits (0: default)
  int persist_chunk = 0;      // iterations a persistent launch runs before returning (0: all)
  int gmres_orth = 0;         // persistent GMRES: 0 modified Gram-Schmidt where it fits, 1 classical
  int persist_launches = 0;   // persistent launches made
  bool alternate = false;     // after each persistent launch, persist_chunk per-step iterations
  int per_step_left = 0;      // per-step iterations still due before the next persistent launch
  bool persistent_now() const { return persistent && per_step_left == 0; }
  void after_persist() {
    if (alternate) per_step_left = persist_chunk;
  }
  void after_step() {
    if (per_step_left > 0) --per_step_left;
  }
  float t_persist_ms = 0.f;   // summed duration of the persistent launches
  int persist_iters = 0;      // iterations they ran
  float t_persist_last_ms = 0.f;
  int persist_last_iters = 0;

  // hands the solve's live mirror to the side thread's cost-aware gate
  void expose(const Mirror* mir) {
    if (ch) ch->live.store(mir, std::memory_order_release);
  }
  void poll(int iter) {
    if (!ch) return;
    const int c = ch->count.load(std::memory_order_acquire);
    if (c <= applied) return;
    std::lock_guard<std::mutex> lock(ch->mu);
    for (int k = applied; k < c; ++k) {
      const int stage = ch->published[k].first;
      cur = ch->published[k].second;
      if (stage >= 0 && stage < 3 && switch_iter[stage] < 0) switch_iter[stage] = iter;
    }
    applied = c;
  }
  // event pairs around every SpMV launch, created in batches (an event
  // creation per launch would cost host time inside the loop)
  void before_spmv(cudaStream_t s) {
    if (!profile) return;
    const size_t need = 2 * (size_t)(n_spmv + 1);
    while (ev.size() < need) {
      for (int q = 0; q < 256; ++q) ev.push_back(ctx->events.take(true));
    }
    CP_CUDA(cudaEventRecord(ev[2 * n_spmv], s));
  }
  void after_spmv(cudaStream_t s) {
    if (!profile) return;
    CP_CUDA(cudaEventRecord(ev[2 * n_spmv + 1], s));
    ++n_spmv;
  }
  float spmv_ms() {
    float tot = 0.f;
    for (int i = 0; i < n_spmv; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) tot += t;
    }
    return tot;
  }
  ~ConfigSource() {
    for (auto e : ev) ctx->events.give(e, true);
  }
};

// How many one-launch-per-step iterations the host keeps queued.  A newly
// published configuration applies only to iterations not yet queued, so while
// the cascade may still publish, the queue holds about kQueueAheadUs of device
// time (at least one iteration, at most depth), from the host's pace while it
// waits for the device (about one iteration's device time per loop).  Slow
// default-kernel iterations (CSR-scalar on power-law rows: hundreds of us)
// then switch within an iteration or two instead of depth; otherwise the
// queue is depth deep.  With one iteration queued the device may idle for the
// host's reaction time between iterations, which costs less than running one
// more slow iteration after a publication.
struct QueueLimit {
  static constexpr double kQueueAheadUs = 300.0;
  int depth, lim;
  bool adapt;
  double ema_us = 0.0;
  std::chrono::steady_clock::time_point last;
  bool have_last = false;
  QueueLimit(int d, bool cascade) : depth(d), lim(cascade ? std::min(2, d) : d), adapt(cascade) {}
  int limit(bool pending) {
    if (!adapt || !pending) return depth;
    return lim;
  }
  void waited() {
    if (!adapt) return;
    const auto now = std::chrono::steady_clock::now();
    if (have_last) {
      const double dt = std::chrono::duration<double, std::micro>(now - last).count();
      ema_us = ema_us > 0.0 ? 0.5 * ema_us + 0.5 * dt : dt;
      const int want = (int)std::ceil(kQueueAheadUs / std::max(ema_us, 1.0));
      lim = std::max(1, std::min(depth, want));
    }
    last = now;
    have_last = true;
  }
};

// Whether this solve has the device to itself as far as the persistent
// kernels go: always, except in a serving lane while another lane holds a job.
static bool device_to_ourselves(const cp_ctx* ctx) {
  return !ctx->lanes_busy || ctx->lanes_busy->load(std::memory_order_acquire) <= 1;
}

// SpMV of the configuration in force (T selects FP64 or FP32 values).
template <typename T>
static int spmv_cur(ConfigSource& cs, const T* x, T* y, const T* dotv, double* part,
                    const int* skip, cudaStream_t s) {
  cs.before_spmv(s);
  const int P = spmv_solver<T>(cs.ctx, cs.m, cs.cur, x, y, dotv, part, skip, s);
  cs.after_spmv(s);
  return P;
}

struct LoopResult {
  int iters = 0;
  int status = CP_OK;
  double res = 0.0;  // last residual norm reported by the device
};

// ------------------------------------------------------------------ CG
// Solves A x = b in precision T from x (x0, or zero when x0_zero).  Stops at
// the recursive residual ||r|| <= tol ||b||; with true_check the FP64 true
// residual is then recomputed and the iteration restarted from x if it is not
// yet below tol (the FP32 inner solves skip that check).
template <typename T>
static LoopResult run_cg(cp_ctx* ctx, ConfigSource& cs, Workspace& ws, const T* b, T* x,
                         bool x0_zero, double tol, int maxit, int depth, bool true_check,
                         double* relres_true) {
  cp_mat* m = cs.m;
  const int64_t n = m->nrows;
  cudaStream_t s = ctx->main;
  auto& B = ws.cg<T>(n);
  T *r = B.r, *p = B.p, *ap = B.ap;
  double *pa = B.pa, *pb = B.pb, *pc = B.pc;
  CgState* st = B.st;
  Mirror* mir = ws.mirror();
  cs.expose(ws.mir);
  CP_CUDA(cudaMemsetAsync(st, 0, sizeof(CgState), s));
  const int persist_iters0 = cs.persist_iters;
  const double tol2 = tol * tol;
  const int G = grid_n(ctx, n);
  // the vector kernels work on pairs in tiles of kBlock * kVecU (update) and
  // twice that (direction); their grids are capped by the resident capacity
  const int Gu = vec_grid(ctx, n, kVecU);
  const int Gd = vec_grid(ctx, n, 2 * kVecU);
  const int* done = &st->done;
  // work on an internal, 16-byte aligned copy of x (the caller's x may be any view)
  T* xw = B.xw;
  CP_CUDA(cudaMemcpyAsync(xw, x, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  T* const x_user = x;
  x = xw;
  LoopResult res;
  int it = 0;
  bool keep_bb = false;
  for (;;) {
    // (re)start: r = b - A x, p = r
    if (!x0_zero || keep_bb) spmv_cur<T>(cs, x, ap, nullptr, nullptr, nullptr, s);
    CP_LAUNCH(ctx, k_cg_init<T>, G, kBlock, 0, s, n, b, (x0_zero && !keep_bb) ? nullptr : ap, r, p,
              pc, pb);
    CP_LAUNCH(ctx, k_cg_init_final, 1, kBlock, 0, s, pc, pb, G, st, it & 1, tol2, mir,
              keep_bb ? 1 : 0);
    keep_bb = true;
    int issued = 0;
    QueueLimit ql(depth, cs.ch != nullptr);
    while (it < maxit) {
      cs.poll(it);
      // The persistent kernel runs only while no prediction work is pending on the
      // side stream: a cooperative grid holds the device, so the side stream's
      // kernels would wait for it.  Until the cascade has finished (or while it
      // only waits on the host), iterations go one launch per step,
      // interleaving with the side kernels.
      const bool side_idle = !cs.ch || cs.ch->finished.load(std::memory_order_acquire) ||
                             cs.ch->side_gpu_idle.load(std::memory_order_acquire);
      if (cs.persistent_now() && side_idle && device_to_ourselves(ctx) &&
          persist_supported<T>(m, cs.cur)) {
        // one cooperative launch runs iterations [it, maxit) until convergence, a
        // breakdown, or the host asks it to return at an iteration boundary
        // because the cascade published a new configuration
        int* yield_d = ws.yield();  // allocates the host-mapped flag on first use
        *(volatile int*)ws.yield_h = 0;
        PersistArgs<T> pa_args;
        pa_args.x = x;
        pa_args.r = r;
        pa_args.p = p;
        pa_args.ap = ap;
        if ((cs.cur.fmt == CP_FMT_HYB && m->hyb_coo.n > 0) || cs.cur.fmt == CP_FMT_COO) {
          if (!B.apc) {  // the kernel leaves it zero after every iteration
            B.apc = ws.get<T>(n);
            CP_CUDA(cudaMemsetAsync(B.apc, 0, n * sizeof(T), s));
          }
          pa_args.apc = B.apc;
        }
        pa_args.pa = pa;
        pa_args.pb = pb;
        pa_args.st = st;
        pa_args.mir = mir;
        pa_args.yield = yield_d;
        pa_args.it0 = it;
        pa_args.itmax = cs.persist_chunk > 0 ? std::min(maxit, it + cs.persist_chunk) : maxit;
        pa_args.tol2 = tol2;
        if (cs.wait_limit_ms > 0.0)
          pa_args.barrier_timeout_ns = (long long)(cs.wait_limit_ms * 1e6);
        cudaEvent_t e0 = ctx->events.take(true), e1 = ctx->events.take(true);
        CP_CUDA(cudaEventRecord(e0, s));
        trace("solve: persistent launch at iteration %d (format %d)", it, cs.cur.fmt);
        persist_launch<T>(ctx, m, cs.cur, pa_args, s, 1);
        ++cs.persist_launches;
        CP_CUDA(cudaEventRecord(e1, s));
        for (;;) {
          const cudaError_t q = cudaEventQuery(e1);
          if (q == cudaSuccess) break;
          if (q != cudaErrorNotReady) CP_CUDA(q);
          // return at the next iteration boundary when a configuration was
          // published, when the side thread needs the GPU again, or when
          // another serving lane got work
          if (!*ws.yield_h &&
              ((cs.ch && (cs.ch->count.load(std::memory_order_acquire) > cs.applied ||
                          (!cs.ch->finished.load(std::memory_order_acquire) &&
                           !cs.ch->side_gpu_idle.load(std::memory_order_acquire)))) ||
               !device_to_ourselves(ctx)))
            *(volatile int*)ws.yield_h = 1;
          std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        float t = 0.f;
        CP_CUDA(cudaEventElapsedTime(&t, e0, e1));
        ctx->events.give(e0, true);
        ctx->events.give(e1, true);
        cs.t_persist_ms += t;
        cs.persist_iters += ws.mir->iters - it;
        cs.t_persist_last_ms = t;
        cs.persist_last_iters = ws.mir->iters - it;
        it = ws.mir->iters;
        trace("solve: persistent launch returned at iteration %d (%.3f ms)", it, t);
        if (ws.mir->done || ws.mir->status != CP_OK) break;
        cs.after_persist();
        continue;  // returned on request: the poll above applies the new configuration
      }
      const int PA = spmv_cur<T>(cs, p, ap, p, pa, done, s);
      CP_LAUNCH(ctx, k_cg_update<T>, Gu, kBlock, 0, s, n, x, r, p, ap, pa, PA, st, it & 1, pb,
                mir);
      CP_LAUNCH(ctx, k_cg_direction<T>, Gd, kBlock, 0, s, n, r, p, pb, Gu, st, it & 1, tol2,
                mir);
      CP_CUDA(cudaEventRecord(ws.event(issued, depth), s));
      ++issued;
      ++it;
      cs.after_step();
      const int lim = ql.limit(cs.ch && !cs.ch->finished.load(std::memory_order_acquire));
      if (issued >= lim) {
        // the one issued lim ago (lim <= depth: its ring slot is not reused yet)
        CP_CUDA(cudaEventSynchronize(ws.event(issued - lim, depth)));
        ql.waited();
        if (ws.mir->done) break;
      }
      // the loop head hands the remaining iterations to the persistent kernel
      // once the side work is over (the queued steps finish first, in stream order)
    }
    CP_CUDA(cudaStreamSynchronize(s));
    res.iters = ws.mir->iters;
    res.status = ws.mir->status;
    res.res = ws.mir->res;
    it = res.iters;
    if (res.status != CP_OK) break;
    if (!true_check) {
      if (!ws.mir->done) res.status = CP_ERR_NOT_CONVERGED;
      break;
    }
    // FP64 true residual b - A x
    spmv_cur<T>(cs, x, ap, nullptr, nullptr, nullptr, s);
    CP_LAUNCH(ctx, k_resid<T>, G, kBlock, 0, s, n, b, ap, (T*)nullptr, pc, (const int*)nullptr);
    double* d_rt = reinterpret_cast<double*>(pa);
    CP_LAUNCH(ctx, k_sum_to, 1, kBlock, 0, s, pc, G, d_rt);
    double rt2 = 0.0, bb = 0.0;
    CP_CUDA(cudaMemcpyAsync(&rt2, d_rt, sizeof(double), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaMemcpyAsync(&bb, &st->bb, sizeof(double), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaStreamSynchronize(s));
    const double rel = bb > 0.0 ? std::sqrt(rt2 / bb) : 0.0;
    if (relres_true) *relres_true = rel;
    if (rel <= tol) break;
    if (it >= maxit) {
      res.status = CP_ERR_NOT_CONVERGED;
      break;
    }
    x0_zero = false;  // restart from the current x
  }
  CP_CUDA(cudaMemcpyAsync(x_user, xw, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  CP_CUDA(cudaStreamSynchronize(s));
  if (cs.persist_iters > persist_iters0 && trace_on()) {
    // the state (with its timers) is zeroed by every call; the iteration count
    // of the solve accumulates over the inner solves of a refinement
    unsigned long long tn[6];
    CP_CUDA(cudaMemcpy(tn, st->t_ns, sizeof(tn), cudaMemcpyDeviceToHost));
    const double k = 1e-3 / (cs.persist_iters - persist_iters0);
    if (tn[4] == 0 && tn[5] == 0)  // the two-barrier kernel (FP32)
      trace("persistent CG per iteration (us): spmv+direction %.2f bar %.2f update %.2f "
            "bar %.2f", tn[0] * k, tn[1] * k, tn[2] * k, tn[3] * k);
    else
      trace("persistent CG per iteration (us): spmv %.2f bar %.2f update %.2f bar %.2f "
            "direction %.2f bar %.2f", tn[0] * k, tn[1] * k, tn[2] * k, tn[3] * k, tn[4] * k,
            tn[5] * k);
  }
  return res;
}

// ------------------------------------------------------------------ GMRES
template <typename T>
static LoopResult run_gmres(cp_ctx* ctx, ConfigSource& cs, Workspace& ws, const T* b, T* x,
                            bool x0_zero, double tol, int mrest, int maxit, int depth,
                            bool true_check, double* relres_true) {
  cp_mat* m = cs.m;
  const int64_t n = m->nrows;
  cudaStream_t s = ctx->main;
  const int64_t ldv = (n + 31) / 32 * 32;
  auto& B = ws.gm<T>(n, ldv, mrest);
  T *V = B.V, *tmp = B.tmp;
  double *part = B.part, *pn = B.pn;
  GmState* st = B.st;
  Mirror* mir = ws.mirror();
  cs.expose(ws.mir);
  CP_CUDA(cudaMemsetAsync(st, 0, sizeof(GmState), s));
  const int persist_iters0 = cs.persist_iters;
  const double tol2 = tol * tol;
  const int G = grid_n(ctx, n);
  // the multi-dot kernel keeps several accumulators a thread: its grid is
  // what stays resident (more blocks would only queue in waves)
  int Gd = G;
  {
    int per_sm = 0;
    CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gm_dots<T>, kBlock, 0));
    const int res = ctx->num_sms * (per_sm > 0 ? per_sm : 1);
    if (Gd > res) Gd = res;
  }
  // ||b||^2 into h1[0] for the first cycle start
  {
    const int P = dot_partials<T>(ctx, n, b, b, pn, nullptr, s);
    CP_LAUNCH(ctx, k_sum_to, 1, kBlock, 0, s, pn, P, &st->h1[0]);
  }
  LoopResult res;
  int first = 1;
  bool finished = false;  // the persistent kernel ended the solve (converged or failed)
  for (;;) {
    // cycle start: V0 = b - A x, beta = ||V0||, V0 /= beta
    int P0 = G;
    if (x0_zero && first) {
      CP_CUDA(cudaMemcpyAsync(V, b, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
      P0 = dot_partials<T>(ctx, n, b, b, pn, nullptr, s);
    } else {
      spmv_cur<T>(cs, x, tmp, nullptr, nullptr, &st->done, s);
      CP_LAUNCH(ctx, k_resid<T>, G, kBlock, 0, s, n, b, tmp, V, pn, &st->done);
    }
    CP_LAUNCH(ctx, k_gm_start, 1, kBlock, 0, s, pn, P0, st, tol2, mir, first);
    CP_LAUNCH(ctx, k_gm_scale<T>, G, kBlock, 0, s, n, V, st, 1);
    first = 0;
    CP_CUDA(cudaStreamSynchronize(s));
    res.iters = ws.mir->iters;
    res.status = ws.mir->status;
    res.res = ws.mir->res;
    if (ws.mir->done || res.status != CP_OK) break;
    if (res.iters >= maxit) {
      res.status = CP_ERR_NOT_CONVERGED;
      break;
    }
    int steps = std::min(mrest, maxit - res.iters);  // this cycle's length
    int issued = 0;
    QueueLimit ql(depth, cs.ch != nullptr);
    bool x_updated = false;  // the persistent kernel ended the cycle and updated x
    int j = 0;
    while (j < steps) {
      cs.poll(res.iters + j);
      // Once no prediction work is pending on the side stream, one cooperative
      // launch takes over the steps (across cycles) until the solve ends, the
      // budget is spent, or the host asks it to return at a step boundary
      // because a new configuration was published or the side needs the GPU.
      const bool side_idle = !cs.ch || cs.ch->finished.load(std::memory_order_acquire) ||
                             cs.ch->side_gpu_idle.load(std::memory_order_acquire);
      if (cs.persistent_now() && side_idle && device_to_ourselves(ctx) &&
          gm_persist_supported<T>(m, cs.cur, mrest)) {
        int* yield_d = ws.yield();
        *(volatile int*)ws.yield_h = 0;
        ws.mir->exit_kind = 0;
        GmPersistArgs<T> ga;
        ga.V = V;
        ga.ldv = ldv;
        ga.x = x;
        ga.b = b;
        ga.part = part;
        ga.part2 = B.part2;
        ga.pn = pn;
        ga.st = st;
        ga.mir = mir;
        ga.yield = yield_d;
        ga.itmax = maxit;
        ga.mrest = mrest;
        ga.mcyc = steps;
        ga.chunk = cs.persist_chunk;
        ga.mgs = cs.gmres_orth == 0 ? 1 : 0;  // a request; the launch checks that it fits
        ga.true_check = true_check ? 1 : 0;
        ga.always_reorth = std::is_same<T, float>::value ? 1 : 0;
        ga.tol2 = tol2;
        if (cs.wait_limit_ms > 0.0)
          ga.barrier_timeout_ns = (long long)(cs.wait_limit_ms * 1e6);
        if ((cs.cur.fmt == CP_FMT_HYB && m->hyb_coo.n > 0) || cs.cur.fmt == CP_FMT_COO) {
          if (!B.wc) {  // the kernel leaves it zero after every product
            B.wc = ws.get<T>(n);
            CP_CUDA(cudaMemsetAsync(B.wc, 0, n * sizeof(T), s));
          }
          ga.wc = B.wc;
        }
        const int it_before = res.iters + j;
        cudaEvent_t e0 = ctx->events.take(true), e1 = ctx->events.take(true);
        CP_CUDA(cudaEventRecord(e0, s));
        trace("solve: persistent GMRES launch at step %d of the cycle (format %d)", j,
              cs.cur.fmt);
        gm_persist_launch<T>(ctx, m, cs.cur, ga, s);
        ++cs.persist_launches;
        CP_CUDA(cudaEventRecord(e1, s));
        for (;;) {
          const cudaError_t q = cudaEventQuery(e1);
          if (q == cudaSuccess) break;
          if (q != cudaErrorNotReady) CP_CUDA(q);
          if (!*ws.yield_h &&
              ((cs.ch && (cs.ch->count.load(std::memory_order_acquire) > cs.applied ||
                          (!cs.ch->finished.load(std::memory_order_acquire) &&
                           !cs.ch->side_gpu_idle.load(std::memory_order_acquire)))) ||
               !device_to_ourselves(ctx)))
            *(volatile int*)ws.yield_h = 1;
          std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        float t = 0.f;
        CP_CUDA(cudaEventElapsedTime(&t, e0, e1));
        ctx->events.give(e0, true);
        ctx->events.give(e1, true);
        const int kind = ws.mir->exit_kind;
        const int ran = ws.mir->iters - it_before;
        cs.t_persist_ms += t;
        cs.persist_iters += ran;
        cs.t_persist_last_ms = t;
        cs.persist_last_iters = ran;
        trace("solve: persistent GMRES returned (kind %d) after %d steps (%.3f ms)", kind, ran, t);
        if (ws.mir->done || ws.mir->status != CP_OK) {
          finished = true;
          break;
        }
        cs.after_persist();
        if (kind == 2) {  // at the end of a cycle, x updated
          x_updated = true;
          break;
        }
        if (kind == 0) break;  // the cycle had ended in a step queued before the launch
        // inside a cycle (possibly a later one): the per-step kernels carry on
        res.iters = ws.mir->iters - ws.mir->jdone;
        steps = ws.mir->mcyc;
        j = ws.mir->jdone;
        issued = 0;
        continue;
      }
      T* vj = V + (int64_t)j * ldv;
      T* w = V + (int64_t)(j + 1) * ldv;
      spmv_cur<T>(cs, vj, w, nullptr, nullptr, &st->halt, s);
      // classical Gram-Schmidt, and a second time only where the first pass
      // removed most of w (k_gm_reorth_test)
      for (int pass = 0; pass < 2; ++pass) {
        double* h = pass == 0 ? st->h1 : st->h2;
        CP_LAUNCH(ctx, k_gm_dots<T>, Gd, kBlock, 0, s, n, V, ldv, j + 1, w, part, st,
                  pass == 0 ? 1 : 0);
        CP_LAUNCH(ctx, k_gm_reduce, pass == 0 ? j + 2 : j + 1, kBlock, 0, s, part, Gd, h, st,
                  pass);
        CP_LAUNCH(ctx, k_gm_sub<T>, G, kBlock, 0, s, n, V, ldv, j + 1, w, h, pn, st, pass);
        if (pass == 0)
          CP_LAUNCH(ctx, k_gm_reorth_test, 1, kBlock, 0, s, pn, G, st, j + 1,
                    std::is_same<T, float>::value ? 1 : 0);
      }
      CP_LAUNCH(ctx, k_gm_givens, 1, kBlock, 0, s, pn, G, st, j, steps, tol2, mir);
      CP_LAUNCH(ctx, k_gm_scale<T>, G, kBlock, 0, s, n, w, st, 1);
      CP_CUDA(cudaEventRecord(ws.event(issued, depth), s));
      ++issued;
      ++j;
      cs.after_step();
      const int lim = ql.limit(cs.ch && !cs.ch->finished.load(std::memory_order_acquire));
      if (issued >= lim) {
        CP_CUDA(cudaEventSynchronize(ws.event(issued - lim, depth)));
        ql.waited();
        if (ws.mir->halt) break;
      }
    }
    if (finished) {
      res.iters = ws.mir->iters;
      res.status = ws.mir->status;
      res.res = ws.mir->res;
      break;
    }
    if (!x_updated) {
      CP_LAUNCH(ctx, k_gm_backsub, 1, 1, 0, s, st);
      CP_LAUNCH(ctx, k_gm_update_x<T>, G, kBlock, 0, s, n, V, ldv, x, st);
    }
    CP_CUDA(cudaStreamSynchronize(s));
    res.iters = ws.mir->iters;
    res.status = ws.mir->status;
    if (res.status != CP_OK) break;
    if (!true_check && ws.mir->conv_est) break;
  }
  if (cs.persist_iters > persist_iters0 && trace_on()) {
    unsigned long long tn[6];
    CP_CUDA(cudaStreamSynchronize(s));
    CP_CUDA(cudaMemcpy(tn, st->t_ns, sizeof(tn), cudaMemcpyDeviceToHost));
    const double k = 1e-3 / (cs.persist_iters - persist_iters0);
    trace("persistent GMRES per step (us): %.2f %.2f %.2f %.2f %.2f %.2f (classical: SpMV + "
          "dots, barrier, subtraction, barrier, second pass, cycle ends; modified: SpMV + first "
          "dots, Givens, columns, -, -, cycle ends)", tn[0] * k, tn[1] * k, tn[2] * k, tn[3] * k, tn[4] * k,
          tn[5] * k);
  }
  if (true_check) {
    // FP64 true residual of the returned x
    spmv_cur<T>(cs, x, tmp, nullptr, nullptr, nullptr, s);
    CP_LAUNCH(ctx, k_resid<T>, G, kBlock, 0, s, n, b, tmp, (T*)nullptr, pn, (const int*)nullptr);
    CP_LAUNCH(ctx, k_sum_to, 1, kBlock, 0, s, pn, G, &st->h2[0]);
    double rt2 = 0.0, bb = 0.0;
    CP_CUDA(cudaMemcpyAsync(&rt2, &st->h2[0], sizeof(double), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaMemcpyAsync(&bb, &st->bb, sizeof(double), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaStreamSynchronize(s));
    const double rel = bb > 0.0 ? std::sqrt(rt2 / bb) : 0.0;
    if (relres_true) *relres_true = rel;
    if (res.status == CP_OK && rel > tol) res.status = CP_ERR_NOT_CONVERGED;
  }
  return res;
}

// ------------------------------------------------------------------ iterative refinement
// x0 = the caller's x.  Loop: r = b - A x in FP64 with the configuration in
// force; stop at ||r|| <= tol ||b||; else solve A d = r in FP32 (values and r
// rounded to nearest), starting from d = 0, and x += d.  The inner solve runs
// to relative max(inner_tol, theta tol ||b|| / ||r||): it stops at inner_tol,
// or once its residual is theta tol ||b||, a correction that already brings the
// outer residual under the target (up to FP32 rounding of A and r).
static LoopResult run_ir(cp_ctx* ctx, ConfigSource& cs, Workspace& ws, const double* b,
                         double* x, double tol, double inner_tol, double theta, int max_outer,
                         int maxit, int depth, bool gmres, int mrest, double* relres,
                         int* outer_out) {
  cp_mat* m = cs.m;
  const int64_t n = m->nrows;
  cudaStream_t s = ctx->main;
  double* r = ws.get<double>(n);
  double* ax = ws.get<double>(n);
  float* r32 = ws.get<float>(n);
  float* d32 = ws.get<float>(n);
  double* part = ws.get<double>(kMaxPartials);
  double* sums = ws.get<double>(2);
  const int G = grid_n(ctx, n);
  double bb = 0.0;
  {
    const int P = dot_partials<double>(ctx, n, b, b, part, nullptr, s);
    CP_LAUNCH(ctx, k_sum_to, 1, kBlock, 0, s, part, P, sums);
    CP_CUDA(cudaMemcpyAsync(&bb, sums, sizeof(double), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaStreamSynchronize(s));
  }
  LoopResult res;
  int outer = 0, inner_total = 0;
  for (;;) {
    cs.poll(inner_total);
    spmv_cur<double>(cs, x, ax, nullptr, nullptr, nullptr, s);
    CP_LAUNCH(ctx, k_resid<double>, G, kBlock, 0, s, n, b, ax, r, part, (const int*)nullptr);
    CP_LAUNCH(ctx, k_sum_to, 1, kBlock, 0, s, part, G, sums + 1);
    double rr = 0.0;
    CP_CUDA(cudaMemcpyAsync(&rr, sums + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaStreamSynchronize(s));
    const double rel = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    *relres = rel;
    res.res = std::sqrt(rr);
    if (!std::isfinite(rel)) {
      res.status = CP_ERR_BREAKDOWN;
      break;
    }
    if (rel <= tol) break;
    if (outer >= max_outer || inner_total >= maxit) {
      res.status = CP_ERR_NOT_CONVERGED;
      break;
    }
    CP_LAUNCH(ctx, (k_cast<double, float>), G, kBlock, 0, s, n, r, r32);
    CP_CUDA(cudaMemsetAsync(d32, 0, n * sizeof(float), s));
    const double itol = std::max(inner_tol, theta * tol / rel);
    LoopResult in = gmres ? run_gmres<float>(ctx, cs, ws, r32, d32, true, itol, mrest,
                                             maxit - inner_total, depth, false, nullptr)
                          : run_cg<float>(ctx, cs, ws, r32, d32, true, itol,
                                          maxit - inner_total, depth, false, nullptr);
    inner_total += in.iters;
    if (in.status == CP_ERR_BREAKDOWN) {
      res.status = CP_ERR_BREAKDOWN;
      break;
    }
    CP_LAUNCH(ctx, k_add_f32, G, kBlock, 0, s, n, x, d32);
    ++outer;
  }
  res.iters = inner_total;
  *outer_out = outer;
  return res;
}

// ------------------------------------------------------------------ entry
void solve(cp_ctx* ctx, cp_mat* m, const double* b, double* x, const cp_solve_opts* o,
           cp_solve_info* info, bool gmres) {
  const auto t0 = Clock::now();
  cp_solve_opts opt;
  cp_solve_opts_default(&opt);
  if (o) opt = *o;
  CP_REQUIRE(opt.tol > 0.0 && opt.maxit >= 0, CP_ERR_INVALID, "tol must be > 0, maxit >= 0");
  CP_REQUIRE(!gmres || (opt.restart >= 1 && opt.restart <= kMaxRestart), CP_ERR_INVALID,
             "GMRES restart must be in 1..%d", kMaxRestart);
  CP_REQUIRE(opt.precision == CP_PREC_FP64 || opt.precision == CP_PREC_FP32_IR, CP_ERR_INVALID,
             "unknown precision %d", opt.precision);
  CP_REQUIRE(opt.ir_theta >= 0.0 && opt.ir_theta < 1.0, CP_ERR_INVALID,
             "ir_theta must be in [0, 1)");
  CP_REQUIRE(opt.mode >= CP_MODE_PLAIN && opt.mode <= CP_MODE_ASYNC, CP_ERR_INVALID,
             "unknown mode %d", opt.mode);
  CP_REQUIRE(m->nrows == m->ncols, CP_ERR_INVALID, "solvers need a square matrix");
  const bool fp32 = opt.precision == CP_PREC_FP32_IR;
  const int depth = opt.check_every > 0 ? opt.check_every : 8;
  const int64_t launches0 = ctx->launches.load();

  ConfigSource cs;
  cs.ctx = ctx;
  cs.m = m;
  cs.fp32 = fp32;
  cs.profile = opt.profile != 0;
  CP_REQUIRE(opt.iteration_kernel >= 0 && opt.iteration_kernel <= 2, CP_ERR_INVALID,
             "iteration_kernel must be 0, 1 or 2");
  CP_REQUIRE(opt.iteration_kernel != 2 || opt.persist_chunk > 0, CP_ERR_INVALID,
             "iteration_kernel 2 needs persist_chunk > 0");
  cs.persistent = opt.iteration_kernel != 1;
  cs.alternate = opt.iteration_kernel == 2;
  CP_REQUIRE(opt.wait_limit_ms >= 0.0, CP_ERR_INVALID, "wait_limit_ms must be >= 0");
  cs.wait_limit_ms = opt.wait_limit_ms;
  CP_REQUIRE(opt.persist_chunk >= 0, CP_ERR_INVALID, "persist_chunk must be >= 0");
  cs.persist_chunk = opt.persist_chunk;
  CP_REQUIRE(opt.gmres_orth == 0 || opt.gmres_orth == 1, CP_ERR_INVALID,
             "gmres_orth must be 0 or 1");
  cs.gmres_orth = opt.gmres_orth;
  cp_config_default(&cs.cur);
  if (opt.force) cs.cur = *opt.force;
  ensure_format(ctx, m, cs.cur, ctx->main);
  if (fp32) ensure_val32(ctx, m, cs.cur, ctx->main);

  Channel ch;
  ch.need_fp32 = fp32;
  // the gate follows an FP64 solve's residuals while it runs (asynchronous
  // mode); the sequential mode predicts before there is any
  ch.tol = (!fp32 && opt.mode == CP_MODE_ASYNC) ? opt.tol : 0.0;
  bool side_posted = false;
  const bool predict = !opt.force && opt.mode != CP_MODE_PLAIN;
  trace("solve: start n=%lld mode=%d precision=%d", (long long)m->nrows, opt.mode, opt.precision);
  if (predict) {
    cs.ch = &ch;
    if (opt.mode == CP_MODE_SEQUENTIAL) {
      run_cascade(ctx, m, ctx->side, &ch);  // predict first, then solve (SerGMRES)
      cs.poll(0);
    } else {
      ctx->side_worker->post([ctx, m, &ch]() { run_cascade(ctx, m, ctx->side, &ch); });
      side_posted = true;
    }
  }
  auto stop_side = [&]() {
    ch.solve_done.store(true);
    ch.cancel.store(true);
    if (side_posted) ctx->side_worker->wait();
    side_posted = false;
  };

  LoopResult res;
  double relres = 0.0;
  int outer = 0;
  Workspace ws(ctx);
  try {
    if (!fp32) {
      res = gmres ? run_gmres<double>(ctx, cs, ws, b, x, false, opt.tol, opt.restart, opt.maxit,
                                      depth, true, &relres)
                  : run_cg<double>(ctx, cs, ws, b, x, false, opt.tol, opt.maxit, depth, true,
                                   &relres);
    } else {
      res = run_ir(ctx, cs, ws, b, x, opt.tol, opt.inner_tol, opt.ir_theta, opt.max_outer,
                   opt.maxit, depth, gmres, opt.restart, &relres, &outer);
    }
    CP_CUDA(cudaStreamSynchronize(ctx->main));
  } catch (...) {
    stop_side();
    throw;
  }
  const float t_total = (float)ms_since(t0);
  stop_side();
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = res.iters;
    info->outer_iters = outer;
    for (int k = 0; k < 3; ++k) info->switch_iter[k] = cs.switch_iter[k];
    info->relres_true = relres;
    info->final_cfg = cs.cur;
    info->t_features_ms = ch.t_features_ms;
    for (int k = 0; k < 3; ++k) info->t_predict_ms[k] = ch.t_predict_ms[k];
    info->t_convert_ms = ch.t_convert_ms;
    info->t_total_ms = t_total;
    info->t_spmv_ms = cs.spmv_ms();
    info->n_spmv = cs.n_spmv;
    info->t_persist_ms = cs.t_persist_ms;
    info->persist_iters = cs.persist_iters;
    info->t_persist_last_ms = cs.t_persist_last_ms;
    info->persist_last_iters = cs.persist_last_iters;
    info->gate_declined = ch.gate_declined;
    info->gate_remaining = ch.gate_remaining;
    info->gate_cost_spmvs = ch.gate_cost;
    info->side_status = ch.status;
    info->persist_launches = cs.persist_launches;
    info->n_launches = (int32_t)(ctx->launches.load() - launches0);
    info->status = res.status;
  }
  if (res.status != CP_OK) {
    if (res.status == CP_ERR_NOT_CONVERGED)
      set_error("not converged: relative residual %.3e after %d iterations", relres, res.iters);
    else if (res.status == CP_ERR_BREAKDOWN)
      set_error("breakdown (non-SPD matrix for CG, or a non-finite value)");
    throw Error{(cp_status)res.status};
  }
}

}  // namespace cp
