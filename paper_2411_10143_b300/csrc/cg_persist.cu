// Persistent CG: every iteration of the conjugate-gradient loop (Sec. I) in
// one cooperative launch.  The grid is the device's resident capacity; three
// phases per iteration are separated by grid-wide barriers instead of kernel
// boundaries:
//   1. Ap = A p with the format's row loop, and the block partials of (p, Ap)
//   2. alpha = (r, r)/(Ap, p) (every block sums the partials in the same order);
//      x += alpha p, r -= alpha Ap, block partials of (r, r)
//   3. beta = (r+, r+)/(r, r); stop if ||r+|| <= tol ||b||; else p = r + beta p
// The host asks the kernel to return at the next iteration boundary (to switch
// to a newly predicted SpMV configuration) through a host-mapped flag that
// block 0 reads in phase 2 and publishes to every block through the state.
// The launch is cooperative, so every block is resident.  The grid barrier is
// the library's own (an arrival counter and a generation word) with a time
// limit: a wait that exceeds it records CP_ERR_TIMEOUT, and every block leaves
// the loop at its next barrier; the iteration loop is bounded by itmax.
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

// Grid-wide barrier with a time limit.  Returns false (in every thread of the
// block) when the wait gave up or another block already did.
__device__ __forceinline__ bool grid_barrier(CgState* st, long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &st->bar_gen;
    volatile int* err = &st->bar_err;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(&st->bar_count, 1u) + 1u;
    int good = 1;
    if (arrived == gridDim.x) {
      st->bar_count = 0;
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        if (*err) {
          good = 0;
          break;
        }
        if ((long long)(global_ns() - t0) > timeout_ns) {
          atomicExch(&st->bar_err, 1);
          good = 0;
          break;
        }
        __nanosleep(8);
      }
    }
    __threadfence();
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

template <typename T, int F, int TPV>
__global__ void __launch_bounds__(kPersistBlock, 1) k_cg_persist(PersistArgs<T> a) {
  // already converged (by iterations queued before this launch): nothing to do
  if (ld_cg(&a.st->done)) return;
  __shared__ double red[40];
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
  unsigned long long tmark = lead ? global_ns() : 0;
  auto lap = [&](int k) {  // block 0's step timer
    if (lead) {
      const unsigned long long now = global_ns();
      st->t_ns[k] += now - tmark;
      tmark = now;
    }
  };
  for (int it = a.it0; it < a.itmax; ++it) {
    const int slot = it & 1;
    // ---- phase 1: Ap = A p, partials of (p, Ap)
    {
      const T acc = spmv_phase<T, F, TPV>(a, so);
      const double s = block_sum((double)acc, red);
      if (threadIdx.x == 0) a.pa[blockIdx.x] = s;
    }
    lap(0);
    if (!grid_barrier(st, a.barrier_timeout_ns)) break;
    lap(1);
    // ---- phase 2: alpha; x += alpha p; r -= alpha Ap; partials of (r, r)
    const double pap = reduce_partials_cg(a.pa, gridDim.x, red);
    const double rr = ld_cg(&st->rr[slot]);
    if (!(pap > 0.0) || !isfinite(pap)) {  // A not SPD, or overflow / NaN: every block stops
      if (lead) {
        st->status = CP_ERR_BREAKDOWN;
        st->done = 1;
        a.mir->status = CP_ERR_BREAKDOWN;
        a.mir->done = 1;
      }
      break;
    }
    const T alpha = (T)(rr / pap);
    {
      V* x2 = reinterpret_cast<V*>(a.x);
      V* r2 = reinterpret_cast<V*>(a.r);
      const V* p2 = reinterpret_cast<const V*>(a.p);
      const V* q2 = reinterpret_cast<const V*>(a.ap);
      T acc = 0;
      for (int64_t i = tid; i < n2; i += stride) {
        const V xv = ld_cg(x2 + i), rv = ld_cg(r2 + i), pv = ld_cg(p2 + i), qv = ld_cg(q2 + i);
        V xn, rn;
        xn.x = fma(alpha, pv.x, xv.x);
        xn.y = fma(alpha, pv.y, xv.y);
        rn.x = fma(-alpha, qv.x, rv.x);
        rn.y = fma(-alpha, qv.y, rv.y);
        x2[i] = xn;
        r2[i] = rn;
        acc = fma(rn.x, rn.x, acc);
        acc = fma(rn.y, rn.y, acc);
      }
      if ((a.n & 1) && tid == 0) {
        const int64_t i = a.n - 1;
        a.x[i] = fma(alpha, ld_cg(a.p + i), ld_cg(a.x + i));
        const T ri = fma(-alpha, ld_cg(a.ap + i), ld_cg(a.r + i));
        a.r[i] = ri;
        acc = fma(ri, ri, acc);
      }
      const double s = block_sum((double)acc, red);
      if (threadIdx.x == 0) a.pb[blockIdx.x] = s;
    }
    if (lead) {
      st->pap = pap;
      st->alpha = rr / pap;
      st->stop = *a.yield;  // the host's request, published to all blocks by the barrier
    }
    lap(2);
    if (!grid_barrier(st, a.barrier_timeout_ns)) break;
    lap(3);
    // ---- phase 3: beta; convergence; p = r + beta p
    const double rr_new = reduce_partials_cg(a.pb, gridDim.x, red);
    const bool bad = !isfinite(rr_new);
    const bool conv = rr_new <= a.tol2 * ld_cg(&st->bb);
    if (lead) {
      st->rr[slot ^ 1] = rr_new;
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
    if (conv || bad) break;
    const T beta = (T)(rr_new / rr);
    {
      const V* r2 = reinterpret_cast<const V*>(a.r);
      V* p2 = reinterpret_cast<V*>(a.p);
      for (int64_t i = tid; i < n2; i += stride) {
        const V rv = ld_cg(r2 + i), pv = ld_cg(p2 + i);
        V pn;
        pn.x = fma(beta, pv.x, rv.x);
        pn.y = fma(beta, pv.y, rv.y);
        p2[i] = pn;
      }
      if ((a.n & 1) && tid == 0) a.p[a.n - 1] = fma(beta, ld_cg(a.p + a.n - 1), ld_cg(a.r + a.n - 1));
    }
    const int stop = *(volatile int*)&st->stop;
    if (stop) break;  // every block read the same value after the last barrier
    lap(4);
    if (!grid_barrier(st, a.barrier_timeout_ns)) break;
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
