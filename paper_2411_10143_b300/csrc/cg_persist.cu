// Persistent CG: every iteration of the conjugate-gradient loop (Sec. I) in
// one cooperative launch.  The grid is the device's resident capacity; the
// phases of an iteration are separated by grid-wide barriers instead of kernel
// boundaries.  k_cg_persist (FP64, and HYB's COO tail) takes three phases:
//   1. Ap = A p with the format's row loop, and the block partials of (p, Ap)
//   2. alpha = (r, r)/(Ap, p); r -= alpha Ap, block partials of (r, r)
//   3. beta = (r+, r+)/(r, r); stop if ||r+|| <= tol ||b||; x += alpha p and,
//      unless stopping, p = r + beta p
// x is updated in phase 3 rather than phase 2 so that p is read once for both
// of its uses; the values are the same as with the textbook order.
// k_cg_persist2 (FP32) takes two, described above it.  Every block sums the
// previous phase's partials in the same fixed order, and one thread per block
// forms alpha and beta (FP64 divisions are sequences on the FP64 pipe, the unit
// that bounds this kernel on parts with a reduced FP64 rate).
// The host asks the kernel to return at the next iteration boundary (to switch
// to a newly predicted SpMV configuration) through a host-mapped flag that
// block 0 reads before the SpMV and publishes to every block through the state.
// The launch is cooperative, so every block is resident.  The grid barrier is
// the library's own (a monotone arrival counter, zeroed by the host before the
// launch) with a time limit: a wait that exceeds it records CP_ERR_TIMEOUT,
// and every block leaves the loop at its next barrier; the iteration loop is
// bounded by itmax.
#include "common.cuh"
#include "internal.cuh"
#include "persist.cuh"
#include "spmv_rows.cuh"

namespace cp {

// Pairs handled per thread per trip of the vector loops: all of a trip's
// loads are issued before its stores.
constexpr int kPersistU = 1;

template <typename T, int F, int TPV>
__global__ void __launch_bounds__(kPersistBlock, 1) k_cg_persist(PersistArgs<T> a) {
  // already converged (by iterations queued before this launch): nothing to do
  if (ld_cg(&a.st->done)) return;
  __shared__ double red[kPersistBlock + 4];
  __shared__ double sc_val;  // alpha (phase 2) or beta (phase 3), formed by thread 0
  __shared__ int sc_flag;    // breakdown (phase 2) or stop (phase 3)
  __shared__ int32_t so[F == kPersistDia ? kDiaMax : 1];
  if constexpr (F == kPersistDia) {
    for (int d = threadIdx.x; d < a.ndiag; d += blockDim.x) so[d] = a.offs[d];  // immutable
    __syncthreads();
  }
  using V = typename Vec2<T>::type;
  constexpr int U = kPersistU;
  const int64_t n2 = a.n >> 1;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  CgState* st = a.st;
  unsigned bar_target = 0;
  unsigned long long tmark = lead ? global_ns() : 0;
  auto lap = [&](int k) {  // block 0's step timer
    if (lead) {
      const unsigned long long now = global_ns();
      st->t_ns[k] += now - tmark;
      tmark = now;
    }
  };
  // Thread 0 keeps ||b||^2 and the current (r, r) in shared memory (every
  // block's thread 0 forms the same values from the same partials), so no step
  // waits on an L2 round trip for them.
  __shared__ double bb, rr_cur;
  if (threadIdx.x == 0) {
    bb = ld_cg(&st->bb);
    rr_cur = ld_cg(&st->rr[a.it0 & 1]);
  }
  V* x2 = reinterpret_cast<V*>(a.x);
  V* r2 = reinterpret_cast<V*>(a.r);
  V* p2 = reinterpret_cast<V*>(a.p);
  const V* q2 = reinterpret_cast<const V*>(a.ap);
  V* qc2 = reinterpret_cast<V*>(a.apc);
  for (int it = a.it0; it < a.itmax; ++it) {
    const int slot = it & 1;
    // the host's request, read (host-mapped, a bus round trip) before the SpMV
    // so that phase 2 does not wait for it
    int yield = 0;
    if (lead) yield = *a.yield;
    // ---- phase 1: Ap = A p, partials of (p, Ap)
    {
      T acc = persist_spmv<T, F, TPV, false, true>(a, so, a.p, a.ap, T(1), T(0), a.p);
      if constexpr (F == kPersistHyb) acc += coo_tail_atomic(a, a.p, a.apc);
      const double s = block_sum_lean((double)acc, red);
      if (threadIdx.x == 0) a.pa[blockIdx.x] = s;
    }
    lap(0);
    bar_target += gridDim.x;
    if (!grid_barrier(&st->bar_count, &st->bar_err, bar_target, a.barrier_timeout_ns)) break;
    lap(1);
    // ---- phase 2: alpha; r -= alpha Ap (HYB: Ap = ap + apc, apc zeroed for
    // the next iteration); partials of (r, r)
    if (threadIdx.x < 32) {
      const double pap = warp_partials_cg(a.pa, gridDim.x);
      if (threadIdx.x == 0) {
        const bool bad = !(pap > 0.0) || !isfinite(pap);  // A not SPD, or overflow / NaN
        const double alpha_d = bad ? 0.0 : rr_cur / pap;
        sc_val = alpha_d;
        sc_flag = bad;
        if (lead) {
          if (bad) {
            st->status = CP_ERR_BREAKDOWN;
            st->done = 1;
            a.mir->status = CP_ERR_BREAKDOWN;
            a.mir->done = 1;
          } else {
            st->pap = pap;
            st->alpha = alpha_d;
          }
          st->stop = yield;  // the host's request, published to all blocks by the barrier
        }
      }
    }
    __syncthreads();
    if (sc_flag) break;  // every block saw the same partials
    const double alpha_d = sc_val;
    const T alpha = (T)alpha_d;
    {
      T acc = 0;
      for (int64_t i0 = tid; i0 < n2; i0 += U * stride) {
        V rv[U], qv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t i = i0 + u * stride;
          if (i < n2) {
            rv[u] = ld_cg(r2 + i);
            qv[u] = ld_cg(q2 + i);
            if constexpr (F == kPersistHyb) {
              const V c = ld_cg(qc2 + i);
              qv[u].x += c.x;
              qv[u].y += c.y;
              qc2[i] = V{T(0), T(0)};
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t i = i0 + u * stride;
          if (i < n2) {
            V rn;
            rn.x = fma(-alpha, qv[u].x, rv[u].x);
            rn.y = fma(-alpha, qv[u].y, rv[u].y);
            r2[i] = rn;
            acc = fma(rn.x, rn.x, acc);
            acc = fma(rn.y, rn.y, acc);
          }
        }
      }
      if ((a.n & 1) && tid == 0) {
        const int64_t i = a.n - 1;
        T qi = ld_cg(a.ap + i);
        if constexpr (F == kPersistHyb) {
          qi += ld_cg(a.apc + i);
          a.apc[i] = T(0);
        }
        const T ri = fma(-alpha, qi, ld_cg(a.r + i));
        a.r[i] = ri;
        acc = fma(ri, ri, acc);
      }
      const double s = block_sum_lean((double)acc, red);
      if (threadIdx.x == 0) a.pb[blockIdx.x] = s;
    }
    lap(2);
    bar_target += gridDim.x;
    if (!grid_barrier(&st->bar_count, &st->bar_err, bar_target, a.barrier_timeout_ns)) break;
    lap(3);
    // ---- phase 3: beta; convergence; x += alpha p; p = r + beta p
    // block 0 published the host's request before the barrier; the load is
    // issued here, with the partials', and used at the end of the phase
    const int stop = *(volatile int*)&st->stop;
    if (threadIdx.x < 32) {
      const double rr_new = warp_partials_cg(a.pb, gridDim.x);
      if (threadIdx.x == 0) {
        const bool bad = !isfinite(rr_new);
        const bool conv = rr_new <= a.tol2 * bb;
        const double beta_d = rr_new / rr_cur;
        rr_cur = rr_new;
        sc_val = beta_d;
        sc_flag = conv || bad;
        if (lead) {
          st->rr[slot ^ 1] = rr_new;
          st->beta = beta_d;
          st->iters += 1;
          a.mir->res = sqrt(rr_new);
          a.mir->iters = st->iters;
          if (bad) {
            st->status = CP_ERR_BREAKDOWN;
            a.mir->status = CP_ERR_BREAKDOWN;
          }
          if (conv || bad) {
            st->done = 1;
            a.mir->done = 1;
          }
        }
      }
    }
    __syncthreads();
    const int fin = sc_flag;
    const T beta = (T)sc_val;
    if (fin) {  // last iteration: x only
      for (int64_t i0 = tid; i0 < n2; i0 += U * stride) {
        V xv[U], pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t i = i0 + u * stride;
          if (i < n2) {
            xv[u] = ld_cg(x2 + i);
            pv[u] = ld_cg(p2 + i);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t i = i0 + u * stride;
          if (i < n2) {
            V xn;
            xn.x = fma(alpha, pv[u].x, xv[u].x);
            xn.y = fma(alpha, pv[u].y, xv[u].y);
            x2[i] = xn;
          }
        }
      }
      if ((a.n & 1) && tid == 0) a.x[a.n - 1] = fma(alpha, ld_cg(a.p + a.n - 1), ld_cg(a.x + a.n - 1));
      break;
    }
    for (int64_t i0 = tid; i0 < n2; i0 += U * stride) {
      V xv[U], rv[U], pv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < n2) {
          xv[u] = ld_cg(x2 + i);
          rv[u] = ld_cg(r2 + i);
          pv[u] = ld_cg(p2 + i);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < n2) {
          V xn, pn;
          xn.x = fma(alpha, pv[u].x, xv[u].x);
          xn.y = fma(alpha, pv[u].y, xv[u].y);
          pn.x = fma(beta, pv[u].x, rv[u].x);
          pn.y = fma(beta, pv[u].y, rv[u].y);
          x2[i] = xn;
          p2[i] = pn;
        }
      }
    }
    if ((a.n & 1) && tid == 0) {
      const int64_t i = a.n - 1;
      const T pi = ld_cg(a.p + i);
      a.x[i] = fma(alpha, pi, ld_cg(a.x + i));
      a.p[i] = fma(beta, pi, ld_cg(a.r + i));
    }
    if (stop) break;  // every block read the same value after the last barrier
    lap(4);
    bar_target += gridDim.x;
    if (!grid_barrier(&st->bar_count, &st->bar_err, bar_target, a.barrier_timeout_ns)) break;
    lap(5);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && *(volatile int*)&st->bar_err) {
    st->status = CP_ERR_TIMEOUT;
    st->done = 1;
    a.mir->status = CP_ERR_TIMEOUT;
    a.mir->done = 1;
  }
}

// Two grid barriers an iteration.  The product of the next direction with A
// comes from A p+ = A r+ + beta A p (exact in exact arithmetic), so the
// direction update joins the SpMV, which reads r+ (complete after the barrier
// that ends the r update) instead of p+:
//   A. beta = (r+, r+)/(r, r); stop if ||r+|| <= tol ||b||; in every row of
//      the format's mapping q_i = (A r+)_i + beta q_i and p_i = r+_i + beta p_i;
//      block partials of (p, q).  A launch's first iteration forms q = A p.
//   B. alpha = (r, r)/(p, q); x += alpha p; r -= alpha q; partials of (r, r)
// q is the one vector carried by a recurrence (a pipelined CG carries three),
// and (p, q) is still formed directly.  The recurrence costs a multiply-add a
// row, which the FP32 inner solves can afford; it ends where the three-phase
// kernel ends (x, r, p and the state alike at a convergence, a breakdown, the
// host's request or itmax).  Not for HYB's COO tail, whose atomics would race
// with the fused row updates.
template <typename T, int F, int TPV>
__global__ void __launch_bounds__(kPersistBlock, 1) k_cg_persist2(PersistArgs<T> a) {
  static_assert(F != kPersistHyb, "the COO tail takes the three-phase kernel");
  if (ld_cg(&a.st->done)) return;
  __shared__ double red[kPersistBlock + 4];
  __shared__ double sc_val;  // alpha (phase B) or beta (phase A), formed by thread 0
  __shared__ int sc_flag;    // breakdown (phase B) or stop (phase A)
  __shared__ int32_t so[F == kPersistDia ? kDiaMax : 1];
  if constexpr (F == kPersistDia) {
    for (int d = threadIdx.x; d < a.ndiag; d += blockDim.x) so[d] = a.offs[d];  // immutable
    __syncthreads();
  }
  using V = typename Vec2<T>::type;
  const int64_t n2 = a.n >> 1;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  CgState* st = a.st;
  unsigned bar_target = 0;
  unsigned long long tmark = lead ? global_ns() : 0;
  auto lap = [&](int k) {  // block 0's step timer
    if (lead) {
      const unsigned long long now = global_ns();
      st->t_ns[k] += now - tmark;
      tmark = now;
    }
  };
  __shared__ double bb, rr_cur;
  if (threadIdx.x == 0) {
    bb = ld_cg(&st->bb);
    rr_cur = ld_cg(&st->rr[a.it0 & 1]);
  }
  V* x2 = reinterpret_cast<V*>(a.x);
  V* r2 = reinterpret_cast<V*>(a.r);
  V* p2 = reinterpret_cast<V*>(a.p);
  const V* q2 = reinterpret_cast<const V*>(a.ap);
  T beta = 0;
  for (int it = a.it0;; ++it) {
    if (it > a.it0) {
      // ---- the end of iteration it - 1: beta; convergence
      // block 0 published the host's request before the last barrier
      const int stop = *(volatile int*)&st->stop;
      if (threadIdx.x < 32) {
        const double rr_new = warp_partials_cg(a.pb, gridDim.x);
        if (threadIdx.x == 0) {
          const bool bad = !isfinite(rr_new);
          const bool conv = rr_new <= a.tol2 * bb;
          const double beta_d = rr_new / rr_cur;
          rr_cur = rr_new;
          sc_val = beta_d;
          sc_flag = conv || bad;
          if (lead) {
            st->rr[((it - 1) & 1) ^ 1] = rr_new;
            st->beta = beta_d;
            st->iters += 1;
            a.mir->res = sqrt(rr_new);
            a.mir->iters = st->iters;
            if (bad) {
              st->status = CP_ERR_BREAKDOWN;
              a.mir->status = CP_ERR_BREAKDOWN;
            }
            if (conv || bad) {
              st->done = 1;
              a.mir->done = 1;
            }
          }
        }
      }
      __syncthreads();
      beta = (T)sc_val;
      if (sc_flag) break;  // x and r are final
      if (stop || it >= a.itmax) {
        // leave p = r + beta p, as the three-phase kernel does
        for (int64_t i = tid; i < n2; i += stride) {
          const V rv = ld_cg(r2 + i), pv = ld_cg(p2 + i);
          p2[i] = V{fma(beta, pv.x, rv.x), fma(beta, pv.y, rv.y)};
        }
        if ((a.n & 1) && tid == 0)
          a.p[a.n - 1] = fma(beta, ld_cg(a.p + a.n - 1), ld_cg(a.r + a.n - 1));
        break;
      }
    } else if (it >= a.itmax) {
      break;
    }
    int yield = 0;
    if (lead) yield = *a.yield;  // host-mapped: read before the SpMV, published in phase B
    // ---- phase A: q = A r + beta q and p = r + beta p (first iteration: q = A p);
    // partials of (p, q)
    {
      T acc;
      if (it == a.it0)
        acc = persist_spmv<T, F, TPV, kRowSolve, true>(a, so, a.p, a.ap, T(1), T(0), a.p);
      else
        acc = persist_spmv<T, F, TPV, kRowCgRec, true>(a, so, a.r, a.ap, T(1), beta, nullptr,
                                                       a.p);
      const double s = block_sum_lean((double)acc, red);
      if (threadIdx.x == 0) a.pa[blockIdx.x] = s;
    }
    lap(0);
    bar_target += gridDim.x;
    if (!grid_barrier(&st->bar_count, &st->bar_err, bar_target, a.barrier_timeout_ns)) break;
    lap(1);
    // ---- phase B: alpha; x += alpha p; r -= alpha q; partials of (r, r)
    if (threadIdx.x < 32) {
      const double pap = warp_partials_cg(a.pa, gridDim.x);
      if (threadIdx.x == 0) {
        const bool bad = !(pap > 0.0) || !isfinite(pap);  // A not SPD, or overflow / NaN
        const double alpha_d = bad ? 0.0 : rr_cur / pap;
        sc_val = alpha_d;
        sc_flag = bad;
        if (lead) {
          if (bad) {
            st->status = CP_ERR_BREAKDOWN;
            st->done = 1;
            a.mir->status = CP_ERR_BREAKDOWN;
            a.mir->done = 1;
          } else {
            st->pap = pap;
            st->alpha = alpha_d;
          }
          st->stop = yield;  // published to all blocks by the barrier
        }
      }
    }
    __syncthreads();
    if (sc_flag) break;  // every block saw the same partials
    const T alpha = (T)sc_val;
    {
      T acc = 0;
      for (int64_t i = tid; i < n2; i += stride) {
        const V xv = ld_cg(x2 + i), pv = ld_cg(p2 + i), rv = ld_cg(r2 + i), qv = ld_cg(q2 + i);
        const V xn{fma(alpha, pv.x, xv.x), fma(alpha, pv.y, xv.y)};
        const V rn{fma(-alpha, qv.x, rv.x), fma(-alpha, qv.y, rv.y)};
        x2[i] = xn;
        r2[i] = rn;
        acc = fma(rn.x, rn.x, acc);
        acc = fma(rn.y, rn.y, acc);
      }
      if ((a.n & 1) && tid == 0) {
        const int64_t i = a.n - 1;
        const T pi = ld_cg(a.p + i);
        a.x[i] = fma(alpha, pi, ld_cg(a.x + i));
        const T ri = fma(-alpha, ld_cg(a.ap + i), ld_cg(a.r + i));
        a.r[i] = ri;
        acc = fma(ri, ri, acc);
      }
      const double s = block_sum_lean((double)acc, red);
      if (threadIdx.x == 0) a.pb[blockIdx.x] = s;
    }
    lap(2);
    bar_target += gridDim.x;
    if (!grid_barrier(&st->bar_count, &st->bar_err, bar_target, a.barrier_timeout_ns)) break;
    lap(3);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && *(volatile int*)&st->bar_err) {
    st->status = CP_ERR_TIMEOUT;
    st->done = 1;
    a.mir->status = CP_ERR_TIMEOUT;
    a.mir->done = 1;
  }
}

// The kernel of an element type and format: two barriers an iteration
// (k_cg_persist2) for FP32, the refinement's inner solves; three (k_cg_persist)
// for FP64, whose loop the FP64 pipe bounds: there the recurrence's extra
// multiply-add a row costs more than the saved barrier (3D Poisson 128^3, DIA:
// 62.0 against 59.8 us an iteration; FP32 27.5 against 30.1 us).  HYB with a
// COO part and COO take three in both precisions.
template <typename T, int F, int TPV>
static auto cg_kernel() {
  if constexpr (sizeof(T) == 4 && F != kPersistHyb) return k_cg_persist2<T, F, TPV>;
  else return k_cg_persist<T, F, TPV>;
}

// ------------------------------------------------------------------ host
template <typename T, int F, int TPV>
static void launch_one(cp_ctx* ctx, PersistArgs<T>& a, cudaStream_t s, int share) {
  auto kern = cg_kernel<T, F, TPV>();
  int per_sm = 0;
  CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersistBlock, 0));
  CP_REQUIRE(per_sm >= 1, CP_ERR_CUDA, "persistent CG kernel does not fit an SM");
  // share = 2: leave half of every SM to concurrent side-stream work
  if (share == 2) per_sm = per_sm > 1 ? per_sm / 2 : 1;
  int grid = ctx->num_sms * per_sm;
  if (grid > kMaxPartials) grid = kMaxPartials;
  void* args[] = {&a};
  // the barrier's arrival counter counts up from zero in every launch
  CP_CUDA(cudaMemsetAsync(&a.st->bar_count, 0, sizeof(unsigned), s));
  CP_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid),
                                      dim3(kPersistBlock), args, 0, s));
  ctx->launches.fetch_add(1, std::memory_order_relaxed);
}

template <typename T>
bool persist_supported(const cp_mat* m, const cp_config& c) {
  return persist_format_ok(m, c, true);
}

template <typename T>
void persist_launch(cp_ctx* ctx, cp_mat* m, const cp_config& c, PersistArgs<T> a,
                    cudaStream_t s, int share) {
  persist_dispatch<T, true>(m, c, a, [&](auto f, auto tpv) {
    launch_one<T, decltype(f)::value, decltype(tpv)::value>(ctx, a, s, share);
  });
}

template bool persist_supported<double>(const cp_mat*, const cp_config&);
template bool persist_supported<float>(const cp_mat*, const cp_config&);
template void persist_launch<double>(cp_ctx*, cp_mat*, const cp_config&, PersistArgs<double>,
                                     cudaStream_t, int);
template void persist_launch<float>(cp_ctx*, cp_mat*, const cp_config&, PersistArgs<float>,
                                    cudaStream_t, int);

}  // namespace cp
