// Shared declarations of the persistent Krylov kernels (cg_persist.cu,
// gm_persist.cu) and their host drivers (krylov.cu): the CG state, the
// host-mapped mirror, the grid barrier and the SpMV phase over the formats a
// persistent kernel runs.  GMRES's own state is in gm_state.cuh.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "internal.cuh"
#include "spmv_rows.cuh"

namespace cp {

struct CgState {
  double rr[2];  // (r, r) of the current iteration, by parity
  double pap, alpha, beta, bb, relres;
  int done;      // recursive residual reached tol (or breakdown): stop
  int status;    // CP_OK / CP_ERR_BREAKDOWN / CP_ERR_TIMEOUT
  int iters;     // completed iterations
  int stop;      // persistent kernel: return at the end of this iteration
  unsigned bar_count;  // arrivals at the persistent kernel's grid barriers (this launch)
  int bar_err;                  // a barrier wait gave up
  // block 0's time in the persistent kernel's steps (ns): SpMV, barrier, update,
  // barrier, direction, barrier
  unsigned long long t_ns[6];
};

constexpr int kPersistBlock = 1024;  // one block per SM: 148 barrier arrivals, 148 partials;
                                     // a multiple of 128 (block_sum_lean)

// Host-mapped mirror written by the kernels that finish an iteration.
struct Mirror {
  volatile double res;    // latest residual norm (recursive / estimated / true)
  volatile double res0;   // residual norm at the (re)start
  volatile double bnorm;  // ||b||
  volatile int done, halt, status, iters, jdone, conv_est;
  volatile int mcyc;       // GMRES: length of the current cycle
  volatile int exit_kind;  // persistent GMRES: 1 = returned inside a cycle (columns
                           // normalised), 2 = returned at a cycle end (x updated)
};

enum {
  kPersistCsrScalar = 0,
  kPersistCsrVector = 1,
  kPersistEll = 2,
  kPersistSell = 3,
  kPersistDia = 4,
  kPersistHyb = 5  // HYB with a COO part (ELL rows plus the COO tail), or COO (no ELL part)
};

// ------------------------------------------------------------------ grid barrier
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

// Grid-wide barrier with a time limit over a monotone arrival counter (zeroed
// by the host before the launch).  target: the arrival count that ends this
// barrier (the block's running count of barriers times the grid size).
// Returns false (in every thread of the block) when the wait gave up or
// another block already did (err set).
__device__ __forceinline__ bool grid_barrier(unsigned* count, int* err, unsigned target,
                                             long long timeout_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* e = err;
    red_add_release(count, 1u);
    int good = 1;
    if ((int)(ld_acquire(count) - target) < 0) {
      const unsigned long long t0 = global_ns();
      while ((int)(ld_acquire(count) - target) < 0) {
        if (*e) {
          good = 0;
          break;
        }
        if ((long long)(global_ns() - t0) > timeout_ns) {
          atomicExch(err, 1);
          good = 0;
          break;
        }
      }
    }
    ok = good && !*e;
  }
  __syncthreads();
  return ok != 0;
}

// ------------------------------------------------------------------ matrix of a persistent kernel
template <typename T>
struct PersistMat {
  int64_t n = 0;
  // CSR
  const int32_t *rp = nullptr, *ci = nullptr;
  const T* v = nullptr;
  // ELL, or HYB's ELL part (K = 0 for COO)
  int64_t K = 0, ld = 0;
  const int32_t* ec = nullptr;
  const T* ev = nullptr;
  // SELL
  int64_t nchunks = 0;
  const int32_t *perm = nullptr, *clen = nullptr;
  const int64_t* cptr = nullptr;
  const int32_t* sc = nullptr;
  const T* sv = nullptr;
  // DIA
  int ndiag = 0;
  const int32_t* offs = nullptr;
  const T* dv = nullptr;
  // HYB's COO part (entries beyond the ELL width, in row order)
  int64_t coo_n = 0;
  const int32_t *coo_row = nullptr, *coo_col = nullptr;
  const T* coo_val = nullptr;
  int coo_vec = 0;  // all three 16-byte aligned: vector loads of 8 entries
};

// y = alpha A x + beta y (GEN = kRowGen) or y = A x (kRowSolve) over the rows
// of the format's grid-stride mapping; returns the thread's share of (A x, dotv)
// when DOT.  GEN = kRowCgRec: the two-barrier CG kernel's fused direction step
// (spmv_rows.cuh), pw being p.  x is never read through the read-only path (the
// persistent kernels rewrite it between phases; ld_x).
template <typename T, int F, int TPV, int GEN, bool DOT>
__device__ __forceinline__ T persist_spmv(const PersistMat<T>& a, const int32_t* so,
                                          const T* x, T* y, T alpha, T beta, const T* dotv,
                                          T* pw = nullptr) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if constexpr (F == kPersistCsrScalar)
    return csr_scalar_rows<T, GEN, DOT, true>(a.n, a.rp, a.ci, a.v, x, y, alpha, beta, dotv,
                                              tid, stride, pw);
  else if constexpr (F == kPersistCsrVector)
    return csr_vector_rows<T, TPV, GEN, DOT, true>(a.n, a.rp, a.ci, a.v, x, y, alpha, beta,
                                                   dotv, tid >> 5, stride >> 5, pw);
  else if constexpr (F == kPersistEll || F == kPersistHyb)  // (HYB: the ELL rows here)
    return ell_rows<T, GEN, DOT, true>(a.n, a.K, a.ld, a.ec, a.ev, x, y, alpha, beta, dotv, tid,
                                       stride, pw);
  else if constexpr (F == kPersistSell)
    return sell_chunks<T, GEN, DOT, true>(a.n, a.nchunks, a.perm, a.clen, a.cptr, a.sc, a.sv, x,
                                          y, alpha, beta, dotv, tid >> 5, stride >> 5, pw);
  else
    return dia_rows<T, GEN, DOT, true>(a.n, a.n, a.ndiag, so, a.dv, x, y, alpha, beta, dotv,
                                       tid, stride, pw);
}

// HYB's COO tail in a persistent SpMV phase: yc[row] += val * x[col] for every
// tail entry, through FP64 (FP32) atomics.  The entries are in row order.  A
// warp takes a tile of 32 * kCooTailE consecutive entries, each lane
// kCooTailE consecutive ones: a lane sums its entries row by row with one FMA
// each and adds a row that starts and ends inside it at once; the rows that
// cross lanes are combined by a segmented scan of the lanes' last partial sums
// and added once per row and tile.  On parts with a reduced FP64 rate the FP64
// instructions bound this loop, and a lane per entry (a product, a scan of five
// additions and a dot-product FMA for every 32 entries) spent about three times
// as many as this.  DOT: returns the thread's share of
// sum_e x[row_e] val_e x[col_e], the tail's part of (x, A x).  yc must not be
// the ELL part's output (other blocks add to any row while the ELL rows are
// stored).
constexpr int kCooTailE = 8;

template <typename T, bool DOT = true>
__device__ __forceinline__ T coo_tail_atomic(const PersistMat<T>& a, const T* x, T* yc) {
  constexpr int E = kCooTailE;
  static_assert(E == 8, "the vector loads take 8 entries");
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  T dot = 0;
  for (int64_t e0 = gw * 32 * E; e0 < a.coo_n; e0 += nw * 32 * E) {
    const int64_t el = e0 + (int64_t)lane * E;  // this lane's first entry
    const int64_t left = a.coo_n - el;
    const int mine = left <= 0 ? 0 : (left < E ? (int)left : E);
    int32_t r[E], c[E];
    T v[E];
    if (mine == E && a.coo_vec) {
      ld8_ro(a.coo_row + el, r);
      ld8_ro(a.coo_col + el, c);
      ld8_ro(a.coo_val + el, v);
    } else {
      // a lane's missing entries repeat its last row with a zero value, and a
      // lane without entries has a negative row of its own, never flushed
#pragma unroll
      for (int u = 0; u < E; ++u) {
        const bool in = u < mine;
        r[u] = in ? __ldg(a.coo_row + el + u) : (u > 0 ? r[u - 1] : -1 - lane);
        c[u] = in ? __ldg(a.coo_col + el + u) : -1;
        v[u] = in ? __ldg(a.coo_val + el + u) : T(0);
      }
    }
    T xg[E];
#pragma unroll
    for (int u = 0; u < E; ++u) xg[u] = c[u] >= 0 ? ld_x<true>(x + c[u]) : T(0);
    const int32_t first = r[0];
    int32_t cur = first;
    T run = 0, head = 0;
    bool split = false;  // a row ended inside this lane
#pragma unroll
    for (int u = 0; u < E; ++u) {
      if (u > 0 && r[u] != cur) {
        if (split) {  // the row lies inside this lane: its whole tail part
          atomicAdd(yc + cur, run);
          if (DOT) dot = fma(ld_cg(x + cur), run, dot);
        } else {
          head = run;  // the lane's first row, which may continue from the left
        }
        split = true;
        cur = r[u];
        run = 0;
      }
      run = fma(v[u], xg[u], run);
    }
    // segmented inclusive scan of the lanes' last partial sums: a run of lanes
    // starts at a lane whose last row began inside it or differs from the
    // previous lane's last row
    const int32_t prev_cur = __shfl_up_sync(full, cur, 1);
    T sv = run;
    bool f = lane == 0 || split || prev_cur != cur;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      if (__all_sync(full, f)) break;  // every run is complete
      const T up = __shfl_up_sync(full, sv, o);
      const bool fup = __shfl_up_sync(full, (int)f, o) != 0;
      if (lane >= o) {
        if (!f) sv += up;
        f = f || fup;
      }
    }
    const T sv_prev = __shfl_up_sync(full, sv, 1);
    const int32_t next_first = __shfl_down_sync(full, first, 1);
    if (split && first >= 0) {  // the first row ends here: add the lanes before with that row
      const T cs = head + (lane > 0 && prev_cur == first ? sv_prev : T(0));
      atomicAdd(yc + first, cs);
      if (DOT) dot = fma(ld_cg(x + first), cs, dot);
    }
    if (cur >= 0 && (lane == 31 || next_first != cur)) {  // the last lane of a run
      atomicAdd(yc + cur, sv);
      if (DOT) dot = fma(ld_cg(x + cur), sv, dot);
    }
  }
  return dot;
}

template <typename T>
struct PersistVals;
template <>
struct PersistVals<double> {
  static const double* csr(const cp_mat* m) { return m->val; }
  static const double* ell(const EllPart& e) { return e.val; }
  static const double* sell(const SellPart& s) { return s.val; }
  static const double* dia(const DiaPart& d) { return d.val; }
  static const double* coo(const CooPart& c) { return c.val; }
};
template <>
struct PersistVals<float> {
  static const float* csr(const cp_mat* m) { return m->val32; }
  static const float* ell(const EllPart& e) { return e.val32; }
  static const float* sell(const SellPart& s) { return s.val32; }
  static const float* dia(const DiaPart& d) { return d.val32; }
  static const float* coo(const CooPart& c) { return c.val32; }
};

// Formats a persistent kernel runs: CSR (scalar or vector), ELL, HYB without a
// COO part (which is ELL), SELL and DIA; with coo_tail, HYB with a COO part and
// COO too (kPersistHyb: the caller's kernel adds the entries by atomics).
inline bool persist_format_ok(const cp_mat* m, const cp_config& c, bool coo_tail = false) {
  if (c.fmt == CP_FMT_CSR) return c.algo == CP_ALGO_SCALAR || c.algo == CP_ALGO_VECTOR;
  if (c.fmt == CP_FMT_HYB) return m->hyb_coo.n == 0 || coo_tail;
  if (c.fmt == CP_FMT_COO) return coo_tail;
  return c.fmt == CP_FMT_ELL || c.fmt == CP_FMT_SELL || c.fmt == CP_FMT_DIA;
}

template <int V>
using IntC = std::integral_constant<int, V>;

// The COO entries a kPersistHyb kernel adds by atomics (row order).
template <typename T>
void persist_tail(PersistMat<T>& a, int64_t n, const int32_t* row, const int32_t* col,
                  const T* val) {
  a.coo_n = n;
  a.coo_row = row;
  a.coo_col = col;
  a.coo_val = val;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  a.coo_vec = al16(row) && al16(col) && al16(val);
}

// Fills a's format fields from m's data for configuration c and calls
// launch(IntC<F>{}, IntC<TPV>{}) with the matching kernel variant.  TAIL: the
// caller's kernel handles HYB's COO part (kPersistHyb).
template <typename T, bool TAIL = false, typename L>
void persist_dispatch(cp_mat* m, const cp_config& c, PersistMat<T>& a, L&& launch) {
  a.n = m->nrows;
  switch (c.fmt) {
    case CP_FMT_CSR:
      a.rp = m->rowptr;
      a.ci = m->col;
      a.v = PersistVals<T>::csr(m);
      if (c.algo == CP_ALGO_SCALAR) {
        launch(IntC<kPersistCsrScalar>{}, IntC<1>{});
      } else {
        switch (c.tpv) {
          case 2: launch(IntC<kPersistCsrVector>{}, IntC<2>{}); break;
          case 4: launch(IntC<kPersistCsrVector>{}, IntC<4>{}); break;
          case 8: launch(IntC<kPersistCsrVector>{}, IntC<8>{}); break;
          case 16: launch(IntC<kPersistCsrVector>{}, IntC<16>{}); break;
          default: launch(IntC<kPersistCsrVector>{}, IntC<32>{}); break;
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
      if (c.fmt == CP_FMT_HYB && m->hyb_coo.n > 0) {
        if constexpr (TAIL) {
          persist_tail(a, m->hyb_coo.n, m->hyb_coo.row, m->hyb_coo.col,
                       PersistVals<T>::coo(m->hyb_coo));
          launch(IntC<kPersistHyb>{}, IntC<1>{});
        } else {
          CP_REQUIRE(false, CP_ERR_UNSUPPORTED, "no persistent kernel for HYB with a COO part");
        }
      } else {
        launch(IntC<kPersistEll>{}, IntC<1>{});
      }
      break;
    }
    case CP_FMT_COO:
      // HYB with an empty ELL part: every entry is in the tail
      if constexpr (TAIL) {
        a.K = 0;
        a.ld = m->nrows;
        persist_tail(a, m->nnz, m->coo.row, m->col, PersistVals<T>::csr(m));
        launch(IntC<kPersistHyb>{}, IntC<1>{});
      } else {
        CP_REQUIRE(false, CP_ERR_UNSUPPORTED, "no persistent kernel for COO");
      }
      break;
    case CP_FMT_SELL:
      a.nchunks = m->sell.nchunks;
      a.perm = m->sell.sigma > 1 ? m->sell.perm : nullptr;
      a.clen = m->sell.chunk_len;
      a.cptr = m->sell.chunk_ptr;
      a.sc = m->sell.col;
      a.sv = PersistVals<T>::sell(m->sell);
      launch(IntC<kPersistSell>{}, IntC<1>{});
      break;
    case CP_FMT_DIA:
      a.ndiag = (int)m->dia.ndiag;
      a.offs = m->dia.offs;
      a.dv = PersistVals<T>::dia(m->dia);
      launch(IntC<kPersistDia>{}, IntC<1>{});
      break;
    default:
      CP_REQUIRE(false, CP_ERR_UNSUPPORTED, "no persistent kernel for format %d", c.fmt);
  }
}

// ------------------------------------------------------------------ CG
template <typename T>
struct PersistArgs : PersistMat<T> {
  T *x = nullptr, *r = nullptr, *p = nullptr, *ap = nullptr;
  T* apc = nullptr;  // HYB / COO: the COO entries' part of Ap, zero between iterations
  double *pa = nullptr, *pb = nullptr;  // block partials, capacity >= grid
  CgState* st = nullptr;
  Mirror* mir = nullptr;
  const volatile int* yield = nullptr;  // host-mapped: return at the next iteration boundary
  int it0 = 0, itmax = 0;
  double tol2 = 0.0;
  long long barrier_timeout_ns = 2000000000ll;
};

template <typename T>
bool persist_supported(const cp_mat* m, const cp_config& c);
// share = 1: the whole device; 2: half of every SM, leaving room for the
// side stream's feature / prediction / conversion kernels while they run.
template <typename T>
void persist_launch(cp_ctx* ctx, cp_mat* m, const cp_config& c, PersistArgs<T> a,
                    cudaStream_t s, int share);

}  // namespace cp
