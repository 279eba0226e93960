// Persistent CG: every iteration of the conjugate-gradient loop (Sec. I) in
// one cooperative launch.  The grid is the device's resident capacity; three
// phases per iteration are separated by grid-wide barriers instead of kernel
// boundaries:
//   1. Ap = A p with the format's row loop, and the block partials of (p, Ap)
//   2. alpha = (r, r)/(Ap, p); r -= alpha Ap, block partials of (r, r)
//   3. beta = (r+, r+)/(r, r); stop if ||r+|| <= tol ||b||; x += alpha p and,
//      unless stopping, p = r + beta p
// x is updated in phase 3 rather than phase 2 so that p is read once for both
// of its uses; the values are the same as with the textbook order.  Every
// block sums the previous phase's partials in the same fixed order, and one
// thread per block forms alpha and beta (FP64 divisions are sequences on the
// FP64 pipe, the unit that bounds this kernel on parts with a reduced FP64 rate).
// The host asks the kernel to return at the next iteration boundary (to switch
// to a newly predicted SpMV configuration) through a host-mapped flag that
// block 0 reads in phase 2 and publishes to every block through the state.
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

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Arrival and polling with release / acquire semantics at GPU scope: the
// block's writes (ordered before thread 0 by the preceding __syncthreads) are
// published by the release; the acquire makes the other blocks' writes visible
// before the block's next reads (which go through L2).
__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier with a time limit.  target: the arrival count that ends
// this barrier (the block's running count of barriers times the grid size).
// Returns false (in every thread of the block) when the wait gave up or
// another block already did.
__device__ __forceinline__ bool grid_barrier(CgState* st, unsigned target,
                                             long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* err = &st->bar_err;
    red_add_release(&st->bar_count, 1u);
    int good = 1;
    if ((int)(ld_acquire(&st->bar_count) - target) < 0) {
      const unsigned long long t0 = global_ns();
      while ((int)(ld_acquire(&st->bar_count) - target) < 0) {
        if (*err) {
          good = 0;
          break;
        }
        if ((long long)(global_ns() - t0) > timeout_ns) {
          atomicExch(&st->bar_err, 1);
          good = 0;
          break;
        }
      }
    }
    ok = good && !*err;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T, int F, int TPV>
__device__ __forceinline__ T spmv_phase(const PersistArgs<T>& a, const int32_t* so) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if constexpr (F == kPersistCsrScalar)
    return csr_scalar_rows<T, false, true, true>(a.n, a.rp, a.ci, a.v, a.p, a.ap, T(1), T(0), a.p, tid,
                                           stride);
  else if constexpr (F == kPersistCsrVector)
    return csr_vector_rows<T, TPV, false, true, true>(a.n, a.rp, a.ci, a.v, a.p, a.ap, T(1), T(0), a.p,
                                                tid >> 5, stride >> 5);
  else if constexpr (F == kPersistEll)
    return ell_rows<T, false, true, true>(a.n, a.K, a.ld, a.ec, a.ev, a.p, a.ap, T(1), T(0), a.p, tid,
                                    stride);
  else if constexpr (F == kPersistSell)
    return sell_chunks<T, false, true, true>(a.n, a.nchunks, a.perm, a.clen, a.cptr, a.sc, a.sv, a.p,
                                       a.ap, T(1), T(0), a.p, tid >> 5, stride >> 5);
  else
    return dia_rows<T, false, true, true>(a.n, a.n, a.ndiag, so, a.dv, a.p, a.ap, T(1), T(0), a.p, tid,
                                    stride);
}

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
  V* x2 = reinterpret_cast<V*>(a.x);
  V* r2 = reinterpret_cast<V*>(a.r);
  V* p2 = reinterpret_cast<V*>(a.p);
  const V* q2 = reinterpret_cast<const V*>(a.ap);
  for (int it = a.it0; it < a.itmax; ++it) {
    const int slot = it & 1;
    // ---- phase 1: Ap = A p, partials of (p, Ap)
    {
      const T acc = spmv_phase<T, F, TPV>(a, so);
      const double s = block_sum_lean((double)acc, red);
      if (threadIdx.x == 0) a.pa[blockIdx.x] = s;
    }
    lap(0);
    bar_target += gridDim.x;
    if (!grid_barrier(st, bar_target, a.barrier_timeout_ns)) break;
    lap(1);
    // ---- phase 2: alpha; r -= alpha Ap; partials of (r, r)
    if (threadIdx.x < 32) {
      const double pap = warp_partials_cg(a.pa, gridDim.x);
      if (threadIdx.x == 0) {
        const bool bad = !(pap > 0.0) || !isfinite(pap);  // A not SPD, or overflow / NaN
        const double alpha_d = bad ? 0.0 : ld_cg(&st->rr[slot]) / pap;
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
          st->stop = *a.yield;  // the host's request, published to all blocks by the barrier
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
        const T ri = fma(-alpha, ld_cg(a.ap + i), ld_cg(a.r + i));
        a.r[i] = ri;
        acc = fma(ri, ri, acc);
      }
      const double s = block_sum_lean((double)acc, red);
      if (threadIdx.x == 0) a.pb[blockIdx.x] = s;
    }
    lap(2);
    bar_target += gridDim.x;
    if (!grid_barrier(st, bar_target, a.barrier_timeout_ns)) break;
    lap(3);
    // ---- phase 3: beta; convergence; x += alpha p; p = r + beta p
    if (threadIdx.x < 32) {
      const double rr_new = warp_partials_cg(a.pb, gridDim.x);
      if (threadIdx.x == 0) {
        const bool bad = !isfinite(rr_new);
        const bool conv = rr_new <= a.tol2 * ld_cg(&st->bb);
        const double beta_d = rr_new / ld_cg(&st->rr[slot]);
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
    const int stop = *(volatile int*)&st->stop;
    if (stop) break;  // every block read the same value after the last barrier
    lap(4);
    bar_target += gridDim.x;
    if (!grid_barrier(st, bar_target, a.barrier_timeout_ns)) break;
    lap(5);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && *(volatile int*)&st->bar_err) {
    st->status = CP_ERR_TIMEOUT;
    st->done = 1;
    a.mir->status = CP_ERR_TIMEOUT;
    a.mir->done = 1;
  }
}

// ------------------------------------------------------------------ host
template <typename T, int F, int TPV>
static void launch_one(cp_ctx* ctx, PersistArgs<T>& a, cudaStream_t s, int share) {
  auto kern = k_cg_persist<T, F, TPV>;
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
  if (c.fmt == CP_FMT_CSR) return c.algo == CP_ALGO_SCALAR || c.algo == CP_ALGO_VECTOR;
  if (c.fmt == CP_FMT_HYB) return m->hyb_coo.n == 0;  // HYB without a COO part is ELL
  return c.fmt == CP_FMT_ELL || c.fmt == CP_FMT_SELL || c.fmt == CP_FMT_DIA;
}

template <typename T>
void persist_launch(cp_ctx* ctx, cp_mat* m, const cp_config& c, PersistArgs<T> a,
                    cudaStream_t s, int share) {
  a.n = m->nrows;
  switch (c.fmt) {
    case CP_FMT_CSR:
      a.rp = m->rowptr;
      a.ci = m->col;
      a.v = PersistVals<T>::csr(m);
      if (c.algo == CP_ALGO_SCALAR) {
        launch_one<T, kPersistCsrScalar, 1>(ctx, a, s, share);
      } else {
        switch (c.tpv) {
          case 2: launch_one<T, kPersistCsrVector, 2>(ctx, a, s, share); break;
          case 4: launch_one<T, kPersistCsrVector, 4>(ctx, a, s, share); break;
          case 8: launch_one<T, kPersistCsrVector, 8>(ctx, a, s, share); break;
          case 16: launch_one<T, kPersistCsrVector, 16>(ctx, a, s, share); break;
          default: launch_one<T, kPersistCsrVector, 32>(ctx, a, s, share); break;
        }
      }
      break;
    case CP_FMT_ELL:
    case CP_FMT_HYB: {
      const EllPart& e = c.fmt == CP_FMT_ELL ? m->ell : m->hyb_ell;
      a.K = e.K;
      a.ld = e.ld;
      a.ec = e.col;
      a.ev = PersistVals<T>::ell(e);
      launch_one<T, kPersistEll, 1>(ctx, a, s, share);
      break;
    }
    case CP_FMT_SELL:
      a.nchunks = m->sell.nchunks;
      a.perm = m->sell.sigma > 1 ? m->sell.perm : nullptr;
      a.clen = m->sell.chunk_len;
      a.cptr = m->sell.chunk_ptr;
      a.sc = m->sell.col;
      a.sv = PersistVals<T>::sell(m->sell);
      launch_one<T, kPersistSell, 1>(ctx, a, s, share);
      break;
    case CP_FMT_DIA:
      a.ndiag = (int)m->dia.ndiag;
      a.offs = m->dia.offs;
      a.dv = PersistVals<T>::dia(m->dia);
      launch_one<T, kPersistDia, 1>(ctx, a, s, share);
      break;
    default:
      CP_REQUIRE(false, CP_ERR_UNSUPPORTED, "no persistent CG kernel for format %d", c.fmt);
  }
}

template bool persist_supported<double>(const cp_mat*, const cp_config&);
template bool persist_supported<float>(const cp_mat*, const cp_config&);
template void persist_launch<double>(cp_ctx*, cp_mat*, const cp_config&, PersistArgs<double>,
                                     cudaStream_t, int);
template void persist_launch<float>(cp_ctx*, cp_mat*, const cp_config&, PersistArgs<float>,
                                    cudaStream_t, int);

}  // namespace cp
