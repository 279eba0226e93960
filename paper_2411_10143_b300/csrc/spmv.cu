// The SpMV family (Sec. III-B-2's configuration space, Fig. 2): CSR-scalar,
// CSR-vector with TpV threads per row, merge-path CSR (Merrill and Garland,
// cited in Sec. V-A), ELL, SELL-C-sigma (slicing, Sec. V-A), HYB and COO.
//
// Every kernel is a persistent grid-stride kernel launched with the resident
// grid of the device (a multiple of the SM count), so a fused reduction leaves
// one partial per block and the consumer can sum them in a fixed order.
// Matrix arrays are read with evict-first loads (COO's through the read-only
// path, whose L1 serves the second half of each sector its vector loads touch);
// x is gathered through the read-only path.  T is the value type (double, or float for the FP32 inner
// solves).  No tensor cores: SpMV moves 12 bytes per FP64 non-zero for one
// FMA, far below any tensor-core shape's arithmetic intensity.
#include "common.cuh"
#include "internal.cuh"
#include "spmv_rows.cuh"

namespace cp {

template <bool DOT>
__device__ __forceinline__ void write_partial(double acc, double* partials) {
  if (DOT) {
    __shared__ double red[33];
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

// The row-parallel SpMV kernels: grid-stride wrappers around the row loops of
// spmv_rows.cuh (which the persistent CG kernel runs as its SpMV phase).
template <typename T, bool GEN, bool DOT>
__global__ void __launch_bounds__(kBlock) k_csr_scalar(
    int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const T* __restrict__ v, const T* __restrict__ x, T* __restrict__ y, T alpha, T beta,
    const T* __restrict__ dotv, double* __restrict__ partials, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const T acc = csr_scalar_rows<T, GEN, DOT>(n, rp, ci, v, x, y, alpha, beta, dotv,
                                             blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                                             (int64_t)gridDim.x * blockDim.x);
  write_partial<DOT>((double)acc, partials);
}

template <typename T, int TPV, bool GEN, bool DOT>
__global__ void __launch_bounds__(kBlock) k_csr_vector(
    int64_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const T* __restrict__ v, const T* __restrict__ x, T* __restrict__ y, T alpha, T beta,
    const T* __restrict__ dotv, double* __restrict__ partials, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const T acc = csr_vector_rows<T, TPV, GEN, DOT>(
      n, rp, ci, v, x, y, alpha, beta, dotv, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,
      ((int64_t)gridDim.x * blockDim.x) >> 5);
  write_partial<DOT>((double)acc, partials);
}

// ------------------------------------------------------------------ merge-path CSR
// The merge of the row-end offsets rowptr[1..n] with the non-zero indices
// 0..nnz-1 is cut into tiles of equal length (n + nnz items in total), so a
// 50k-entry row costs the same per item as a 3-entry row.  A tile's start is
// the split point found by a binary search along its diagonal.
//
// Two kernels.  The matrix path (cp_spmv and the solvers) runs warp tiles
// (k_csr_merge_warp below) whose start points k_merge_partition computes once
// per matrix.  The allocation-free entry point has no per-matrix set-up and
// searches in the kernel (tile_start = null), so it runs block tiles
// (k_csr_merge), eight times larger, to spread each search over more
// items.  The block first stages the whole tile in
// shared memory with coalesced loads: the row ends, and for every non-zero of
// the tile its value and the x entry its column selects (the gather of x is
// issued here, all of a thread's loads back to back).  Each thread then walks
// kMergeItems consecutive items out of shared memory (an odd item count keeps
// a half-warp's FP64 reads on distinct banks), one FMA per non-zero.  Rows
// that a thread finishes are written directly; partial rows are combined
// inside the block by a segmented scan, and the partial of the row still open
// at the tile's end becomes the tile's carry, added by k_merge_fixup.

// First split point (i = row ends consumed, k = non-zeros consumed) on diagonal
// d of the merge path, with ties taking the row end after the non-zeros < it.
__device__ __forceinline__ int64_t merge_search(int64_t d, const int32_t* row_end, int64_t n,
                                                int64_t nnz) {
  int64_t lo = d > nnz ? d - nnz : 0;
  int64_t hi = d < n ? d : n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)row_end[mid] <= d - mid - 1) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <typename T, bool GEN>
__global__ void __launch_bounds__(kBlock) k_csr_merge(
    int64_t n, int64_t nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const T* __restrict__ v, const T* __restrict__ x, T* __restrict__ y, T alpha, T beta,
    int64_t ntiles, const int32_t* __restrict__ tile_start, int32_t* __restrict__ carry_row,
    T* __restrict__ carry_val, const int* __restrict__ skip) {
  static_assert(kMergeItems % 2 == 1, "an odd item count keeps the walk's reads conflict-free");
  if (skip && *skip) return;
  __shared__ int32_t s_end[kMergeTile + 1];
  __shared__ T s_val[kMergeTile];   // the tile's values
  __shared__ T s_x[kMergeTile];     // x[col] of each of the tile's non-zeros
  __shared__ int64_t s_bounds[2];
  __shared__ int32_t s_row[kBlock];  // row each thread ends in (its open row)
  __shared__ T s_carry[kBlock];      // sum of that row's partials up to the thread
  __shared__ int32_t s_wfirst[kBlock / 32], s_wlast[kBlock / 32];  // per warp: open rows
  __shared__ T s_wval[kBlock / 32], s_cin[kBlock / 32];              // of lanes 0 and 31
  const int64_t total = n + nnz;
  const int32_t* row_end = rp + 1;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t d0 = t * kMergeTile;
    const int64_t d1 = d0 + kMergeTile < total ? d0 + kMergeTile : total;
    if (tile_start) {
      if (threadIdx.x < 2) s_bounds[threadIdx.x] = tile_start[t + threadIdx.x];
    } else {
      if (threadIdx.x == 0) s_bounds[0] = merge_search(d0, row_end, n, nnz);
      if (threadIdx.x == 32) s_bounds[1] = merge_search(d1, row_end, n, nnz);
    }
    __syncthreads();
    const int64_t i0 = s_bounds[0], i1 = s_bounds[1];
    const int64_t k0 = d0 - i0, k1 = d1 - i1;
    // stage row_end[i0 .. min(i1, n-1)] and the tile's k1 - k0 non-zeros
    // (at most kMergeTile of each: (i1 - i0) + (k1 - k0) = d1 - d0)
    const int64_t last = i1 < n ? i1 : n - 1;
    for (int64_t r = i0 + threadIdx.x; r <= last; r += blockDim.x) s_end[r - i0] = row_end[r];
    {
      const int cnt = (int)(k1 - k0);
      int32_t c[kMergeItems];
      T a[kMergeItems];
#pragma unroll
      for (int q = 0; q < kMergeItems; ++q) {
        const int j = threadIdx.x + q * kBlock;
        if (j < cnt) {
          c[q] = ld_stream(ci + k0 + j);
          a[q] = ld_stream(v + k0 + j);
        }
      }
#pragma unroll
      for (int q = 0; q < kMergeItems; ++q) {
        const int j = threadIdx.x + q * kBlock;
        if (j < cnt) {
          s_val[j] = a[q];
          s_x[j] = ld_ro(x + c[q]);
        }
      }
    }
    __syncthreads();
    // this thread's split inside the tile
    int64_t dt = d0 + (int64_t)threadIdx.x * kMergeItems;
    if (dt > d1) dt = d1;
    // search rows i in [i0, i1] with i + k = dt and k in [k0, d1 - i1]
    int64_t a = dt - k1 > i0 ? dt - k1 : i0;
    int64_t b = dt - k0 < i1 ? dt - k0 : i1;
    while (a < b) {
      const int64_t mid = (a + b) >> 1;
      if ((int64_t)s_end[mid - i0] <= dt - mid - 1) a = mid + 1;
      else b = mid;
    }
    // walk with tile-relative indices: row ri = i - i0, non-zero kk = k - k0
    int ri = (int)(a - i0), kk = (int)(dt - a - k0);
    const int start_ri = ri;
    const int nsteps = (int)((dt + kMergeItems < d1 ? dt + kMergeItems : d1) - dt);
    const int32_t k0i = (int32_t)k0;
    T sum = 0, head = 0;
    bool has_head = false;
    int row_limit = s_end[ri] - k0i;
    for (int q = 0; q < nsteps; ++q) {
      if (kk < row_limit) {
        sum = fma(s_val[kk], s_x[kk], sum);
        ++kk;
      } else {
        if (ri == start_ri) {
          head = sum;
          has_head = true;
        } else {
          store_row<T, GEN>(y, i0 + ri, sum, alpha, beta);
        }
        sum = 0;
        ++ri;
        row_limit = s_end[ri] - k0i;
      }
    }
    // Every thread leaves a partial of the row it ends in (its open row).  An
    // inclusive segmented scan over the block's threads, segments = equal open
    // rows (rows never decrease along the threads, so each segment is a run),
    // gives each thread the sum of its run up to itself: a log-depth scan, where
    // a tile inside one long row would otherwise add 256 partials in sequence.
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t end_row = i0 + ri;
    const int32_t open_row = (int32_t)(end_row < n ? end_row : n);
    T run = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const T up = __shfl_up_sync(0xffffffffu, run, off);
      const int32_t up_row = __shfl_up_sync(0xffffffffu, open_row, off);
      if (lane >= off && up_row == open_row) run += up;
    }
    const int32_t warp_first = __shfl_sync(0xffffffffu, open_row, 0);
    if (lane == 31) {
      s_wlast[wid] = open_row;
      s_wval[wid] = run;
    }
    if (lane == 0) s_wfirst[wid] = open_row;
    __syncthreads();
    if (threadIdx.x == 0) {
      // carry into each warp's first run from the warps before it
      s_cin[0] = 0;
      for (int w = 1; w < kBlock / 32; ++w) {
        const T upto = s_wval[w - 1] + (s_wfirst[w - 1] == s_wlast[w - 1] ? s_cin[w - 1] : T(0));
        s_cin[w] = s_wlast[w - 1] == s_wfirst[w] ? upto : T(0);
      }
    }
    __syncthreads();
    if (open_row == warp_first) run += s_cin[wid];
    s_row[threadIdx.x] = open_row;
    s_carry[threadIdx.x] = run;
    __syncthreads();
    if (has_head) {
      // add the partials of the preceding threads that ended inside start_row
      const int32_t start_row = (int32_t)(i0 + start_ri);
      const T c = threadIdx.x > 0 && s_row[threadIdx.x - 1] == start_row
                      ? s_carry[threadIdx.x - 1] : T(0);
      store_row<T, GEN>(y, start_row, head + c, alpha, beta);
    }
    if (threadIdx.x == blockDim.x - 1) {
      carry_row[t] = open_row < n ? open_row : -1;
      carry_val[t] = run;
    }
    __syncthreads();
  }
}

// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes): the data goes
// to shared memory without passing through registers, and a thread waits for
// its own copies by commit group.
__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_t(T* smem, const T* gmem) {
  if constexpr (sizeof(T) == 8) cp_async_8(smem, gmem);
  else cp_async_4(smem, gmem);
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// waits until at most one committed group of this thread is still in flight
__device__ __forceinline__ void cp_async_wait_prev() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// Bulk asynchronous copies (cp.async.bulk, the TMA engine) into shared memory,
// completed on an mbarrier.  Both addresses 16-byte aligned, size a multiple
// of 16 bytes.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// Waits (bounded) until the phase with the given parity of bar has completed;
// false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (bulk copy) writes
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

constexpr int kMergeWarps = 4;  // warps per block of the warp-tile kernel

// The matrix path's merge-path kernel: warp tiles of kMergeWarpTile items,
// each warp independent of the others (no block barrier), with the tile start
// points computed once per matrix.  Each warp runs a two-stage pipeline over
// its tiles: while it walks one tile out of shared memory, the copies of its
// next tile's row ends, column indices and values are in flight into the
// other half of its shared-memory slice.  The copies are bulk copies on the
// TMA engine (one per array, issued by one lane, 16-byte aligned windows
// around the tile's ranges, completed on the half's mbarrier); an array whose
// rounded window would run past its end (the matrix's last tiles) is copied
// entry by entry with cp.async instead.  Every wait for the copies is bounded:
// one that gives up sets *err (reported as CP_ERR_TIMEOUT at the matrix's next
// merge-path launch) and ends the warp's work.
// Each lane finds its split by a search in the staged row ends and takes the
// next lane's split as its end, so it knows the non-zeros it owns (at most
// kMergeItems, contiguous) and gathers their x entries back to back before
// walking its items.  A warp-wide segmented scan (shuffles) combines the rows
// that cross lanes; the partial of the row open at the tile's end is the
// tile's carry.
template <typename T, bool GEN>
__global__ void __launch_bounds__(32 * kMergeWarps) k_csr_merge_warp(
    int64_t n, int64_t nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
    const T* __restrict__ v, const T* __restrict__ x, T* __restrict__ y, T alpha, T beta,
    int64_t ntiles, const int32_t* __restrict__ tile_start, int32_t* __restrict__ carry_row,
    T* __restrict__ carry_val, const int* __restrict__ skip, int* __restrict__ err) {
  constexpr int W = kMergeWarpTile;
  constexpr int SLOTS = W + 8;  // a tile's 16-byte aligned window of any of the arrays
  if (skip && *skip) return;
  __shared__ __align__(16) int32_t s_end[kMergeWarps][2][SLOTS];
  __shared__ __align__(16) int32_t s_col[kMergeWarps][2][SLOTS];
  __shared__ __align__(16) T s_val[kMergeWarps][2][SLOTS];
  __shared__ __align__(8) uint64_t s_bar[kMergeWarps][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t total = n + nnz;
  const int64_t stride = (int64_t)gridDim.x * kMergeWarps;
  constexpr int64_t VE = 16 / sizeof(T);  // values per 16 bytes
  if (lane == 0) {
    mbar_init(&s_bar[wid][0], 1);
    mbar_init(&s_bar[wid][1], 1);
    mbar_init_fence();
  }
  __syncwarp();
  // A tile's window of each array: [lo, hi) rounded out to 16 bytes.  The
  // row-end window covers rp[i0 + 1 .. last + 1]; the column and value windows
  // the tile's non-zeros [k0, k0 + cnt).
  struct Win {
    int64_t e_lo, e_hi, c_lo, c_hi, v_lo, v_hi;
  };
  auto window = [&](int64_t tt, int32_t a0, int32_t a1, int& cnt, int32_t& k0, int32_t& last) {
    const int64_t d0 = tt * W;
    const int len = (int)(d0 + W < total ? W : total - d0);
    k0 = (int32_t)(d0 - a0);
    cnt = len - (a1 - a0);
    last = a1 < n ? a1 : (int32_t)(n - 1);
    Win wn;
    wn.e_lo = ((int64_t)a0 + 1) & ~int64_t(3);
    wn.e_hi = ((int64_t)last + 2 + 3) & ~int64_t(3);
    wn.c_lo = (int64_t)k0 & ~int64_t(3);
    wn.c_hi = ((int64_t)k0 + cnt + 3) & ~int64_t(3);
    wn.v_lo = (int64_t)k0 & ~(VE - 1);
    wn.v_hi = ((int64_t)k0 + cnt + VE - 1) & ~(VE - 1);
    return wn;
  };
  // issue the copies of tile tt (bounds a0, a1) into half h: a bulk copy per
  // array by lane 0, or, for an array whose rounded window would run past its
  // end (the matrix's last tiles), cp.async copies of the needed entries
  auto stage = [&](int64_t tt, int h, int32_t a0, int32_t a1) {
    int cnt;
    int32_t k0, last;
    const Win wn = window(tt, a0, a1, cnt, k0, last);
    int32_t* e = s_end[wid][h];
    int32_t* c = s_col[wid][h];
    T* w = s_val[wid][h];
    const bool be = wn.e_hi <= n + 1;
    const bool bc = cnt > 0 && wn.c_hi <= nnz;
    const bool bv = cnt > 0 && wn.v_hi <= nnz;
    if (lane == 0) {
      const uint32_t bytes = (be ? (uint32_t)(wn.e_hi - wn.e_lo) * 4u : 0u) +
                             (bc ? (uint32_t)(wn.c_hi - wn.c_lo) * 4u : 0u) +
                             (bv ? (uint32_t)(wn.v_hi - wn.v_lo) * (uint32_t)sizeof(T) : 0u);
      fence_proxy_async();
      mbar_arrive_expect_tx(&s_bar[wid][h], bytes);
      if (be) bulk_g2s(e, rp + wn.e_lo, (uint32_t)(wn.e_hi - wn.e_lo) * 4u, &s_bar[wid][h]);
      if (bc) bulk_g2s(c, ci + wn.c_lo, (uint32_t)(wn.c_hi - wn.c_lo) * 4u, &s_bar[wid][h]);
      if (bv)
        bulk_g2s(w, v + wn.v_lo, (uint32_t)(wn.v_hi - wn.v_lo) * (uint32_t)sizeof(T),
                 &s_bar[wid][h]);
    }
    if (!be)
      for (int32_t r = a0 + lane; r <= last; r += 32)
        cp_async_4(e + (r + 1 - wn.e_lo), rp + r + 1);
    if (!bc || !bv) {
#pragma unroll
      for (int q = 0; q < kMergeItems; ++q) {
        const int j = lane + 32 * q;
        if (j < cnt) {
          if (!bc) cp_async_4(c + (k0 + j - wn.c_lo), ci + k0 + j);
          if (!bv) cp_async_t(w + (k0 + j - wn.v_lo), v + k0 + j);
        }
      }
    }
  };
  uint32_t ph0 = 0u, ph1 = 0u;  // phase parity of each half's mbarrier
  bool ok = true;
  int64_t t = (int64_t)blockIdx.x * kMergeWarps + wid;
  // bounds of the current tile (b0, b1) and of the next one (nb0, nb1)
  int32_t b0 = 0, b1 = 0, nb0 = 0, nb1 = 0;
  if (t < ntiles) {
    b0 = tile_start[t];
    b1 = tile_start[t + 1];
    stage(t, 0, b0, b1);
  }
  cp_async_commit();
  if (t + stride < ntiles) {
    nb0 = tile_start[t + stride];
    nb1 = tile_start[t + stride + 1];
  }
  int h = 0;
  for (; t < ntiles && ok; t += stride, h ^= 1) {
    const int32_t i0 = b0, i1 = b1;
    // the next tile's copies go out before this tile is walked
    if (t + stride < ntiles) stage(t + stride, h ^ 1, nb0, nb1);
    cp_async_commit();  // one group per iteration, possibly empty
    b0 = nb0;
    b1 = nb1;
    if (t + 2 * stride < ntiles) {
      nb0 = tile_start[t + 2 * stride];
      nb1 = tile_start[t + 2 * stride + 1];
    }
    cp_async_wait_prev();  // this tile's element copies have landed (the next ones may not)
    ok = mbar_wait(&s_bar[wid][h], h ? ph1 : ph0);  // and its bulk copies
    if (h) ph1 ^= 1u;
    else ph0 ^= 1u;
    __syncwarp();
    if (!ok) {
      // the copies did not land within the bound: record it (the host reports
      // CP_ERR_TIMEOUT), give the other half's copies a bounded wait, and stop
      if (lane == 0) atomicExch(err, 1);
      if (t + stride < ntiles) (void)mbar_wait(&s_bar[wid][h ^ 1], h ? ph0 : ph1);
      break;
    }
    int cnt_w;
    int32_t k0_w, last_w;
    const Win wn = window(t, i0, i1, cnt_w, k0_w, last_w);
    const int32_t* e_w = s_end[wid][h] + (i0 + 1 - wn.e_lo);
    const int32_t* c_w = s_col[wid][h] + (k0_w - wn.c_lo);
    const T* v_w = s_val[wid][h] + (k0_w - wn.v_lo);
    const int64_t d0 = t * W;
    const int len = (int)(d0 + W < total ? W : total - d0);  // items in the tile
    const int32_t k0 = (int32_t)(d0 - i0);
    const int ni = i1 - i0;    // row ends in the tile
    const int cnt = len - ni;  // non-zeros in the tile
    // this lane's split on its diagonal dr (tile-relative): rows ri_s consumed,
    // non-zeros kk_s consumed, ri_s + kk_s = dr
    const int dr = lane * kMergeItems < len ? lane * kMergeItems : len;
    int a = dr - cnt > 0 ? dr - cnt : 0;
    int b = dr < ni ? dr : ni;
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (e_w[mid] - k0 <= dr - mid - 1) a = mid + 1;
      else b = mid;
    }
    const int ri_s = a;
    const int kk_s = dr - a;
    // the lane's end is the next lane's start (the last lane's: the tile's end)
    int ri_e = __shfl_down_sync(0xffffffffu, ri_s, 1);
    int kk_e = __shfl_down_sync(0xffffffffu, kk_s, 1);
    if (lane == 31) {
      ri_e = ni;
      kk_e = cnt;
    }
    // the lane's non-zeros kk_s .. kk_e - 1: their x gathers back to back
    const int nz = kk_e - kk_s;
    T xv[kMergeItems];
#pragma unroll
    for (int q = 0; q < kMergeItems; ++q)
      if (q < nz) xv[q] = ld_ro(x + c_w[kk_s + q]);
    // walk: before non-zero k, every row whose end is <= k closes
    int ri = ri_s;
    T sum = 0, head = 0;
    bool has_head = false;
#pragma unroll
    for (int q = 0; q < kMergeItems; ++q) {
      if (q < nz) {
        const int32_t kabs = k0 + kk_s + q;
        while (e_w[ri] <= kabs) {
          if (ri == ri_s) {
            head = sum;
            has_head = true;
          } else {
            store_row<T, GEN>(y, i0 + ri, sum, alpha, beta);
          }
          sum = 0;
          ++ri;
        }
        sum = fma(v_w[kk_s + q], xv[q], sum);
      }
    }
    while (ri < ri_e) {  // row ends after the lane's last non-zero
      if (ri == ri_s) {
        head = sum;
        has_head = true;
      } else {
        store_row<T, GEN>(y, i0 + ri, sum, alpha, beta);
      }
      sum = 0;
      ++ri;
    }
    // segmented inclusive scan of the open rows' partials across the warp
    // (FP64 adds cost as much as the walk's FMAs on this GPU, so the scan stops
    // as soon as no run spans more lanes than the steps so far cover: one step
    // when rows cross at most one lane boundary)
    const int32_t open_row = i0 + ri;  // n when the tile ends the matrix
    T run = sum;
    for (int off = 1; off < 32; off <<= 1) {
      const int32_t up_row = __shfl_up_sync(0xffffffffu, open_row, off);
      const bool joins = lane >= off && up_row == open_row;
      if (!__any_sync(0xffffffffu, joins)) break;
      const T up = __shfl_up_sync(0xffffffffu, run, off);
      if (joins) run += up;
    }
    const T prev_run = __shfl_up_sync(0xffffffffu, run, 1);
    const int32_t prev_row = __shfl_up_sync(0xffffffffu, open_row, 1);
    if (has_head) {
      const int32_t start_row = i0 + ri_s;
      const T c = lane > 0 && prev_row == start_row ? prev_run : T(0);
      store_row<T, GEN>(y, start_row, head + c, alpha, beta);
    }
    if (lane == 31) {
      carry_row[t] = open_row < n ? open_row : -1;
      carry_val[t] = run;
    }
    __syncwarp();  // every lane is done with half h before it is restaged
  }
}

// tile_start[t] = first split row of the diagonal t * tile, t = 0..ntiles
__global__ void k_merge_partition(int64_t n, int64_t nnz, const int32_t* __restrict__ rp,
                                  int64_t ntiles, int64_t tile, int32_t* __restrict__ tile_start) {
  const int64_t total = n + nnz;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = t * tile < total ? t * tile : total;
    tile_start[t] = (int32_t)merge_search(d, rp + 1, n, nnz);
  }
}

template <typename T>
__global__ void k_merge_fixup(int64_t ntiles, const int32_t* __restrict__ carry_row,
                              const T* __restrict__ carry_val, T* __restrict__ y, T alpha,
                              const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = carry_row[t];
    if (r >= 0) atomicAdd(y + r, alpha * carry_val[t]);
  }
}

template <typename T, bool GEN, bool DOT>
__global__ void __launch_bounds__(kBlock) k_ell(
    int64_t n, int64_t K, int64_t ld, const int32_t* __restrict__ ec, const T* __restrict__ ev,
    const T* __restrict__ x, T* __restrict__ y, T alpha, T beta, const T* __restrict__ dotv,
    double* __restrict__ partials, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const T acc = ell_rows<T, GEN, DOT>(n, K, ld, ec, ev, x, y, alpha, beta, dotv,
                                      blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                                      (int64_t)gridDim.x * blockDim.x);
  write_partial<DOT>((double)acc, partials);
}

template <typename T, bool GEN, bool DOT>
__global__ void __launch_bounds__(kBlock) k_sell(
    int64_t n, int64_t nchunks, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ clen, const int64_t* __restrict__ cptr,
    const int32_t* __restrict__ sc, const T* __restrict__ sv, const T* __restrict__ x,
    T* __restrict__ y, T alpha, T beta, const T* __restrict__ dotv,
    double* __restrict__ partials, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const T acc = sell_chunks<T, GEN, DOT>(n, nchunks, perm, clen, cptr, sc, sv, x, y, alpha, beta,
                                         dotv, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,
                                         ((int64_t)gridDim.x * blockDim.x) >> 5);
  write_partial<DOT>((double)acc, partials);
}

template <typename T, bool GEN, bool DOT>
__global__ void __launch_bounds__(kBlock) k_dia(
    int64_t n, int64_t ncols, int ndiag, const int32_t* __restrict__ offs,
    const T* __restrict__ dv, const T* __restrict__ x, T* __restrict__ y, T alpha, T beta,
    const T* __restrict__ dotv, double* __restrict__ partials, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ int32_t so[kDiaMax];
  for (int d = threadIdx.x; d < ndiag; d += blockDim.x) so[d] = offs[d];
  __syncthreads();
  const T acc = dia_rows<T, GEN, DOT>(n, ncols, ndiag, so, dv, x, y, alpha, beta, dotv,
                                      blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                                      (int64_t)gridDim.x * blockDim.x);
  write_partial<DOT>((double)acc, partials);
}

// ------------------------------------------------------------------ COO (warp-tiled segmented sums)
// Each warp takes kCooWarpTile consecutive entries (sorted by row); each lane
// loads its kCooItems consecutive entries straight into registers (16-byte
// vector loads through L1, which serves the second half of every sector),
// gathers x for all of them and sums them row by row in a fully unrolled walk
// (one FMA per entry).  (Staging the tile through shared memory for coalesced
// loads left the kernel throttled on the shared-memory pipe.)
// A row inside one lane's entries is written directly.  Rows that span lanes
// are combined with a segmented shuffle scan over the lanes' last segments;
// the lane that holds a row's last entry in the warp writes it, with an atomic
// if the row touches the warp's first or last entry (other warps may hold
// entries of it).  No shared memory and no block barrier: long rows cost the
// same per entry as short ones.  ADD: y already holds the rest of the row
// (beta*y, or HYB's ELL part) and every write adds to it; otherwise y is zero
// and a row completed in one place is stored.
constexpr int kCooItems = 8;
constexpr int kCooWarpTile = 32 * kCooItems;

// ONE: alpha is 1, and a write spends no FP64 instruction (a store, or an
// atomic add, which the L2 performs): on B300 the FP64 pipe, not DRAM, bounds
// this kernel on matrices with short rows.
template <typename T, bool ADD, bool ONE>
__device__ __forceinline__ void coo_put(T* y, int32_t r, T alpha, T s) {
  if constexpr (ONE) {
    if constexpr (ADD) atomicAdd(y + r, s);  // the row is this warp's alone: the same sum
    else y[r] = s;
  } else {
    y[r] = ADD ? fma(alpha, s, y[r]) : alpha * s;
  }
}

template <typename T, bool ADD, bool ONE>
__global__ void __launch_bounds__(kBlock) k_coo(
    int64_t nnz, const int32_t* __restrict__ row, const int32_t* __restrict__ col,
    const T* __restrict__ val, const T* __restrict__ x, T* __restrict__ y, T alpha,
    const int* __restrict__ skip) {
  if (skip && *skip) return;
  static_assert(kCooItems == 8, "the vector loads take 8 entries");
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t ntiles = (nnz + kCooWarpTile - 1) / kCooWarpTile;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  const bool vec = al16(row) && al16(col) && al16(val);
  for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < ntiles;
       t += nwarps) {
    const int64_t e0 = t * kCooWarpTile;
    const int cnt = (int)(nnz - e0 < kCooWarpTile ? nnz - e0 : kCooWarpTile);
    const int j0 = lane * kCooItems;
    const int mine = cnt - j0 < 0 ? 0 : (cnt - j0 < kCooItems ? cnt - j0 : kCooItems);
    int32_t r[kCooItems], c[kCooItems];
    T w[kCooItems], xv[kCooItems];
    if (vec && mine == kCooItems) {
      ld8_ro(row + e0 + j0, r);
      ld8_ro(col + e0 + j0, c);
      ld8_ro(val + e0 + j0, w);
    } else {
#pragma unroll
      for (int u = 0; u < kCooItems; ++u) {
        const bool in = u < mine;
        r[u] = in ? __ldg(row + e0 + j0 + u) : -1;
        c[u] = in ? __ldg(col + e0 + j0 + u) : 0;
        w[u] = in ? __ldg(val + e0 + j0 + u) : T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < kCooItems; ++u) xv[u] = u < mine ? ld_ro(x + c[u]) : T(0);
    const int32_t first = r[0];
    int32_t cur = r[0];
    T head = 0, sum = 0;
    bool multi = false;
#pragma unroll
    for (int u = 0; u < kCooItems; ++u) {
      if (u < mine) {
        if (u > 0 && r[u] != cur) {
          if (!multi) head = sum;  // the first segment closes
          else coo_put<T, ADD, ONE>(y, cur, alpha, sum);  // a row inside this lane only
          multi = true;
          cur = r[u];
          sum = 0;
        }
        sum = fma(w[u], xv[u], sum);
      }
    }
    // segmented inclusive scan of the lanes' last segments: a run starts at a
    // lane whose last segment began inside it (multi), or whose last row
    // differs from the previous lane's
    const int32_t prev_cur = __shfl_up_sync(0xffffffffu, cur, 1);
    T v = sum;
    bool f = lane == 0 || multi || prev_cur != cur;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      if (__all_sync(0xffffffffu, f)) break;  // every run is complete (short rows)
      const T up = __shfl_up_sync(0xffffffffu, v, o);
      const bool fup = __shfl_up_sync(0xffffffffu, (int)f, o) != 0;
      if (lane >= o) {
        if (!f) v += up;
        f = f || fup;
      }
    }
    const T v_prev = __shfl_up_sync(0xffffffffu, v, 1);
    const int32_t next_first = __shfl_down_sync(0xffffffffu, first, 1);
    const int32_t warp_row0 = __shfl_sync(0xffffffffu, first, 0);
    const bool last_in_warp = mine > 0 && j0 + mine == cnt;
    if (multi) {
      // the first row ends in this lane: add the run of preceding lanes' last
      // segments with that row (the scan value of the previous lane)
      const T cs = head + (lane > 0 && prev_cur == first ? v_prev : T(0));
      if (warp_row0 == first) atomicAdd(y + first, ONE ? cs : alpha * cs);  // may start earlier
      else coo_put<T, ADD, ONE>(y, first, alpha, cs);
    }
    if (mine > 0 && (last_in_warp || next_first != cur)) {
      // this lane holds the last entry in the warp of its last row
      if (last_in_warp || warp_row0 == cur) atomicAdd(y + cur, ONE ? v : alpha * v);
      else coo_put<T, ADD, ONE>(y, cur, alpha, v);
    }
  }
}

template <typename T>
__global__ void k_scale(int64_t n, T* __restrict__ y, T beta, const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = beta == T(0) ? T(0) : beta * y[i];
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_dot_partials(int64_t n, const T* __restrict__ a,
                                                         const T* __restrict__ b,
                                                         double* __restrict__ partials,
                                                         const int* __restrict__ skip) {
  if (skip && *skip) return;
  T acc = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(a[i], b[i], acc);
  __shared__ double red[33];
  const double s = block_sum((double)acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// ------------------------------------------------------------------ launchers
template <typename T>
struct Vals;
template <>
struct Vals<double> {
  static const double* dia(const DiaPart& d) { return d.val; }
  static const double* csr(const cp_mat* m) { return m->val; }
  static const double* ell(const EllPart& e) { return e.val; }
  static const double* sell(const SellPart& s) { return s.val; }
  static const double* coo(const CooPart& c) { return c.val; }
};
template <>
struct Vals<float> {
  static const float* dia(const DiaPart& d) { return d.val32; }
  static const float* csr(const cp_mat* m) { return m->val32; }
  static const float* ell(const EllPart& e) { return e.val32; }
  static const float* sell(const SellPart& s) { return s.val32; }
  static const float* coo(const CooPart& c) { return c.val32; }
};

template <typename T, bool GEN, bool DOT>
static void launch_csr_vector(cp_ctx* ctx, int tpv, int grid, cudaStream_t s, int64_t n,
                              const int32_t* rp, const int32_t* ci, const T* v, const T* x, T* y,
                              T alpha, T beta, const T* dotv, double* partials, const int* skip) {
#define CP_VEC_CASE(TPV)                                                                     \
  case TPV:                                                                                  \
    CP_LAUNCH(ctx, (k_csr_vector<T, TPV, GEN, DOT>), grid, kBlock, 0, s, n, rp, ci, v, x, y, \
              alpha, beta, dotv, partials, skip);                                            \
    break;
  switch (tpv) {
    CP_VEC_CASE(2)
    CP_VEC_CASE(4)
    CP_VEC_CASE(8)
    CP_VEC_CASE(16)
    CP_VEC_CASE(32)
    default:
      CP_REQUIRE(false, CP_ERR_UNSUPPORTED, "TpV %d not supported", tpv);
  }
#undef CP_VEC_CASE
}

// Grid for a grid-stride loop over `units` one-thread work units in which
// every thread runs the same number of trips: the resident grid needs
// trips = ceil(units / (grid_stream * kBlock)) of them, and the grid is shrunk
// to the fewest blocks that cover the units in that many trips.  (3.5 trips on
// the full grid would leave half of the threads idle in the last one.)
static int balanced_grid(cp_ctx* ctx, int64_t units) {
  const int64_t per = (int64_t)ctx->grid_stream * kBlock;
  const int64_t trips = units > 0 ? (units + per - 1) / per : 1;
  const int64_t g = (units + trips * kBlock - 1) / (trips * kBlock);
  return (int)(g < 1 ? 1 : g > ctx->grid_stream ? ctx->grid_stream : g);
}

// The row-parallel SpMVs without a fused dot product (CSR-scalar, CSR-vector,
// ELL, HYB's ELL part, DIA): one trip per thread (a row, a row pair, or TPV
// lanes' share of rows), up to the block-partials capacity.  The blocks beyond
// the resident grid keep more loads in flight from the start: uniform 8 per row
// (n 2M) ELL 81.7 -> 72.5 us, CSR-vector4 82.7 -> 79.6 us; banded CSR-scalar
// 234 -> 215 us, CSR-vector4 132 -> 116 us; neutral on the stencils.  (SELL
// keeps the resident grid: one trip each was 5-8 % slower on 3D Poisson.)
// With a fused dot the resident grid stays: every block of the next kernel sums
// one partial per SpMV block.
static int wide_grid(int64_t units) {
  int64_t g = (units + kBlock - 1) / kBlock;
  if (g > kMaxPartials) g = kMaxPartials;
  return (int)(g < 1 ? 1 : g);
}

static int grid_for(cp_ctx* ctx, int64_t work_items) {
  const int64_t need = (work_items + kBlock - 1) / kBlock;
  int64_t g = need < ctx->grid_stream ? need : ctx->grid_stream;
  return (int)(g < 1 ? 1 : g);
}

void merge_partition(cp_ctx* ctx, cp_mat* m, cudaStream_t s) {
  CP_LAUNCH(ctx, k_merge_partition, grid_for(ctx, m->merge_tiles + 1), kBlock, 0, s, m->nrows,
            m->nnz, m->rowptr, m->merge_tiles, (int64_t)kMergeWarpTile, m->merge_start);
}

// The merge-path kernels stage ~20-40 KB of tiles in shared memory:
// prefer the largest shared-memory carve-out so that several blocks share an SM.
void spmv_set_attributes() {
  const int carve = cudaSharedmemCarveoutMaxShared;
  CP_CUDA(cudaFuncSetAttribute(k_csr_merge<double, false>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, carve));
  CP_CUDA(cudaFuncSetAttribute(k_csr_merge_warp<double, false>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, carve));
  CP_CUDA(cudaFuncSetAttribute(k_csr_merge_warp<double, true>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, carve));
  CP_CUDA(cudaFuncSetAttribute(k_csr_merge_warp<float, false>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, carve));
  CP_CUDA(cudaFuncSetAttribute(k_csr_merge_warp<float, true>,
                               cudaFuncAttributePreferredSharedMemoryCarveout, carve));
}

// One wave of the warp-tile merge-path kernel (its shared memory and
// registers bound the blocks an SM holds); each warp takes every
// (gridDim * kMergeWarps)-th warp tile.
template <typename T, bool GEN>
static int merge_warp_grid(int num_sms, int64_t tiles) {
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_csr_merge_warp<T, GEN>,
                                                      32 * kMergeWarps, 0) != cudaSuccess)
      b = 1;
    return b > 0 ? b : 1;
  }();
  int64_t g = (int64_t)num_sms * per_sm;
  const int64_t need = (tiles + kMergeWarps - 1) / kMergeWarps;
  if (g > need) g = need;
  return (int)(g < 1 ? 1 : g);
}

// One wave of the merge-path kernel: its staged tile (about 39 KB of shared
// memory in FP64) bounds the blocks an SM holds; tiles are equal work, so each
// block of the wave takes every gridDim-th tile.
template <typename T, bool GEN>
static int merge_grid(int num_sms, int64_t cap, int64_t tiles) {
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_csr_merge<T, GEN>, kBlock, 0) !=
        cudaSuccess)
      b = 1;
    return b > 0 ? b : 1;
  }();
  int64_t g = (int64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g > tiles) g = tiles;
  return (int)(g < 1 ? 1 : g);
}

// One wave of the COO kernel: its registers (not the thread limit) bound the
// blocks an SM holds, and a second wave would only queue behind the first.
template <typename T, bool ADD, bool ONE>
static int coo_grid(cp_ctx* ctx, int64_t nnz) {
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_coo<T, ADD, ONE>, kBlock, 0) !=
        cudaSuccess)
      b = 1;
    return b > 0 ? b : 1;
  }();
  int64_t cap = (int64_t)ctx->num_sms * per_sm;
  if (cap > ctx->grid_stream) cap = ctx->grid_stream;
  const int64_t tiles = (nnz + kCooWarpTile * (kBlock / 32) - 1) / (kCooWarpTile * (kBlock / 32));
  return (int)(tiles < 1 ? 1 : tiles < cap ? tiles : cap);
}

// y (+)= alpha A x over COO entries (row-sorted), with the alpha == 1 variant
// when it applies.
template <typename T, bool ADD>
static void launch_coo(cp_ctx* ctx, int64_t nnz, const int32_t* row, const int32_t* col,
                       const T* val, const T* x, T* y, T alpha, const int* skip, cudaStream_t s) {
  if (alpha == T(1))
    CP_LAUNCH(ctx, (k_coo<T, ADD, true>), (coo_grid<T, ADD, true>(ctx, nnz)), kBlock, 0, s, nnz,
              row, col, val, x, y, alpha, skip);
  else
    CP_LAUNCH(ctx, (k_coo<T, ADD, false>), (coo_grid<T, ADD, false>(ctx, nnz)), kBlock, 0, s, nnz,
              row, col, val, x, y, alpha, skip);
}

// One routine for both forms: GEN = general alpha/beta, DOT = fused partials.
// skip (device flag, may be null): when set at launch time the kernels return
// at once, so a converged solve's queued iterations cost only their launch.
template <typename T, bool GEN, bool DOT>
static int spmv_dispatch(cp_ctx* ctx, cp_mat* m, const cp_config& cfg, T alpha, const T* x,
                         T beta, T* y, const T* dotv, double* partials, const int* skip,
                         cudaStream_t s) {
  const int64_t n = m->nrows;
  switch (cfg.fmt) {
    case CP_FMT_CSR: {
      const T* v = Vals<T>::csr(m);
      if (cfg.algo == CP_ALGO_VECTOR) {
        const int g = DOT ? balanced_grid(ctx, n * cfg.tpv) : wide_grid(n * cfg.tpv);
        launch_csr_vector<T, GEN, DOT>(ctx, cfg.tpv, g, s, n, m->rowptr, m->col, v, x, y, alpha,
                                       beta, dotv, partials, skip);
        return DOT ? g : 0;
      }
      if (cfg.algo == CP_ALGO_MERGE) {
        // an earlier launch on this matrix whose bounded wait for its tile copies
        // gave up (its y is incomplete) is reported here, at the next launch
        if (m->merge_err && *reinterpret_cast<volatile int*>(m->merge_err)) {
          *reinterpret_cast<volatile int*>(m->merge_err) = 0;
          CP_REQUIRE(false, CP_ERR_TIMEOUT,
                     "an earlier merge-path SpMV on this matrix gave up waiting for its tile "
                     "copies; its result was incomplete");
        }
        const int g = merge_warp_grid<T, GEN>(ctx->num_sms, m->merge_tiles);
        CP_LAUNCH(ctx, (k_csr_merge_warp<T, GEN>), g, 32 * kMergeWarps, 0, s, n, m->nnz, m->rowptr,
                  m->col, v, x, y, alpha, beta, m->merge_tiles, m->merge_start,
                  m->merge_carry_row, reinterpret_cast<T*>(m->merge_carry_val), skip,
                  m->merge_err_dev);
        CP_LAUNCH(ctx, k_merge_fixup<T>, grid_for(ctx, m->merge_tiles), kBlock, 0, s,
                  m->merge_tiles, m->merge_carry_row,
                  reinterpret_cast<const T*>(m->merge_carry_val), y, GEN ? alpha : T(1), skip);
        break;
      }
      const int g = DOT ? balanced_grid(ctx, n) : wide_grid(n);
      CP_LAUNCH(ctx, (k_csr_scalar<T, GEN, DOT>), g, kBlock, 0, s, n, m->rowptr, m->col, v, x, y,
                alpha, beta, dotv, partials, skip);
      return DOT ? g : 0;
    }
    case CP_FMT_ELL: {
      const int g = DOT ? balanced_grid(ctx, (n + 1) / 2) : wide_grid((n + 1) / 2);
      CP_LAUNCH(ctx, (k_ell<T, GEN, DOT>), g, kBlock, 0, s, n, m->ell.K, m->ell.ld, m->ell.col,
                Vals<T>::ell(m->ell), x, y, alpha, beta, dotv, partials, skip);
      return DOT ? g : 0;
    }
    case CP_FMT_SELL: {
      const int g = balanced_grid(ctx, m->sell.nchunks * 32);  // a warp per chunk
      CP_LAUNCH(ctx, (k_sell<T, GEN, DOT>), g, kBlock, 0, s, n, m->sell.nchunks,
                m->sell.sigma > 1 ? m->sell.perm : nullptr, m->sell.chunk_len, m->sell.chunk_ptr,
                m->sell.col, Vals<T>::sell(m->sell), x, y, alpha, beta, dotv, partials, skip);
      return DOT ? g : 0;
    }
    case CP_FMT_HYB: {
      const int g = DOT ? balanced_grid(ctx, (n + 1) / 2) : wide_grid((n + 1) / 2);
      if (m->hyb_coo.n == 0) {  // every row fits the ELL part: the fused ELL kernel suffices
        CP_LAUNCH(ctx, (k_ell<T, GEN, DOT>), g, kBlock, 0, s, n, m->hyb_ell.K, m->hyb_ell.ld,
                  m->hyb_ell.col, Vals<T>::ell(m->hyb_ell), x, y, alpha, beta, dotv, partials,
                  skip);
        return DOT ? g : 0;
      }
      CP_LAUNCH(ctx, (k_ell<T, GEN, false>), g, kBlock, 0, s, n, m->hyb_ell.K, m->hyb_ell.ld,
                m->hyb_ell.col, Vals<T>::ell(m->hyb_ell), x, y, alpha, beta, nullptr, nullptr,
                skip);
      if (m->hyb_coo.n > 0)
        launch_coo<T, true>(ctx, m->hyb_coo.n, m->hyb_coo.row, m->hyb_coo.col,
                            Vals<T>::coo(m->hyb_coo), x, y, GEN ? alpha : T(1), skip, s);
      break;
    }
    case CP_FMT_DIA: {
      const int g = DOT ? balanced_grid(ctx, (n + 1) / 2) : wide_grid((n + 1) / 2);
      CP_LAUNCH(ctx, (k_dia<T, GEN, DOT>), g, kBlock, 0, s, n, m->ncols, (int)m->dia.ndiag,
                m->dia.offs, Vals<T>::dia(m->dia), x, y, alpha, beta, dotv, partials, skip);
      return DOT ? g : 0;
    }
    case CP_FMT_COO: {
      CP_LAUNCH(ctx, k_scale<T>, grid_for(ctx, n), kBlock, 0, s, n, y, GEN ? beta : T(0), skip);
      if (m->nnz > 0 && GEN && beta != T(0))
        launch_coo<T, true>(ctx, m->nnz, m->coo.row, m->col, Vals<T>::csr(m), x, y, alpha, skip,
                            s);
      else if (m->nnz > 0)
        launch_coo<T, false>(ctx, m->nnz, m->coo.row, m->col, Vals<T>::csr(m), x, y,
                             GEN ? alpha : T(1), skip, s);
      break;
    }
    default:
      CP_REQUIRE(false, CP_ERR_UNSUPPORTED, "unknown format %d", cfg.fmt);
  }
  // formats without a fused reduction: a separate pass for the partials
  if (DOT) {
    const int g = grid_for(ctx, n);
    CP_LAUNCH(ctx, k_dot_partials<T>, g, kBlock, 0, s, n, y, dotv, partials, skip);
    return g;
  }
  return 0;
}

template <typename T>
int spmv_solver(cp_ctx* ctx, cp_mat* m, const cp_config& cfg, const T* x, T* y, const T* dotv,
                double* partials, const int* skip, cudaStream_t s) {
  if (dotv)
    return spmv_dispatch<T, false, true>(ctx, m, cfg, T(1), x, T(0), y, dotv, partials, skip, s);
  return spmv_dispatch<T, false, false>(ctx, m, cfg, T(1), x, T(0), y, nullptr, nullptr, skip, s);
}

template <typename T>
void spmv_general(cp_ctx* ctx, cp_mat* m, const cp_config& cfg, T alpha, const T* x, T beta,
                  T* y, cudaStream_t s) {
  // y = A x is the plain form bit for bit (1 * s = s, and beta = 0 never reads
  // y); it saves the scaling and the test of beta, two FP64-pipe operations a
  // row, in kernels the FP64 pipe bounds
  if (alpha == T(1) && beta == T(0))
    spmv_dispatch<T, false, false>(ctx, m, cfg, T(1), x, T(0), y, nullptr, nullptr, nullptr, s);
  else
    spmv_dispatch<T, true, false>(ctx, m, cfg, alpha, x, beta, y, nullptr, nullptr, nullptr, s);
}

template <typename T>
int dot_partials(cp_ctx* ctx, int64_t n, const T* a, const T* b, double* partials,
                 const int* skip, cudaStream_t s) {
  const int g = grid_for(ctx, n);
  CP_LAUNCH(ctx, k_dot_partials<T>, g, kBlock, 0, s, n, a, b, partials, skip);
  return g;
}

template int spmv_solver<double>(cp_ctx*, cp_mat*, const cp_config&, const double*, double*,
                                 const double*, double*, const int*, cudaStream_t);
template int spmv_solver<float>(cp_ctx*, cp_mat*, const cp_config&, const float*, float*,
                                const float*, double*, const int*, cudaStream_t);
template void spmv_general<double>(cp_ctx*, cp_mat*, const cp_config&, double, const double*,
                                   double, double*, cudaStream_t);
template void spmv_general<float>(cp_ctx*, cp_mat*, const cp_config&, float, const float*, float,
                                  float*, cudaStream_t);
template int dot_partials<double>(cp_ctx*, int64_t, const double*, const double*, double*,
                                  const int*, cudaStream_t);
template int dot_partials<float>(cp_ctx*, int64_t, const float*, const float*, double*,
                                 const int*, cudaStream_t);

}  // namespace cp

// ------------------------------------------------------------------ allocation-free entry point
// A merge-path CSR SpMV for callers that cannot allocate device memory (see
// cp_spmv_csr_merge_noalloc in cascade.h).  Its per-tile carry scratch lives in
// these file-scope device arrays, which every GPU that loads the library keeps
// until the process exits.  Host code may not use the array names as device
// addresses: each device's addresses come from cudaGetSymbolAddress below.
namespace cp {

constexpr int64_t kNoAllocMaxTiles = 65536;  // (nrows + nnz) <= 65536 * kMergeTile

static __device__ __align__(256) int32_t g_noalloc_carry_row[kNoAllocMaxTiles];
static __device__ __align__(256) double g_noalloc_carry_val[kNoAllocMaxTiles];

struct NoAllocDevice {
  bool ready = false;
  int32_t* carry_row = nullptr;  // device addresses of the arrays above
  double* carry_val = nullptr;
  int num_sms = 0;
};
static std::mutex g_noalloc_mu;
static NoAllocDevice g_noalloc_dev[64];

// Set-up once per device, with that device current.
static const NoAllocDevice& noalloc_setup(int dev) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.ready) {
    CP_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d.carry_row), g_noalloc_carry_row));
    CP_CUDA(cudaGetSymbolAddress(reinterpret_cast<void**>(&d.carry_val), g_noalloc_carry_val));
    CP_CUDA(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
    spmv_set_attributes();  // function attributes only: allocates nothing
    d.ready = true;
  }
  return d;
}

}  // namespace cp

extern "C" cp_status cp_spmv_csr_merge_noalloc(int64_t nrows, int64_t ncols, int64_t nnz,
                                               const int32_t* rowptr, const int32_t* col,
                                               const double* val, const double* x, double* y,
                                               void* stream) {
  using namespace cp;
  try {
    CP_REQUIRE(rowptr && x && y && (nnz == 0 || (col && val)), CP_ERR_INVALID,
               "cp_spmv_csr_merge_noalloc: NULL pointer argument");
    CP_REQUIRE(nrows >= 1 && ncols >= 1 && nnz >= 0 && nrows < (int64_t(1) << 31) &&
                   nnz < (int64_t(1) << 31),
               CP_ERR_INVALID, "cp_spmv_csr_merge_noalloc: sizes out of range");
    const int64_t tiles = (nrows + nnz + kMergeTile - 1) / kMergeTile;
    CP_REQUIRE(tiles <= kNoAllocMaxTiles, CP_ERR_INVALID,
               "cp_spmv_csr_merge_noalloc: nrows + nnz = %lld exceeds the maximum %lld of its "
               "fixed scratch; use cp_spmv instead",
               (long long)(nrows + nnz), (long long)(kNoAllocMaxTiles * kMergeTile));
    int dev = 0;
    CP_CUDA(cudaGetDevice(&dev));
    CP_REQUIRE(dev >= 0 && dev < 64, CP_ERR_INVALID, "device index %d not supported", dev);
    const NoAllocDevice& d = noalloc_setup(dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t cap = (int64_t)d.num_sms * 8;
    const int grid = merge_grid<double, false>(d.num_sms, cap, tiles);
    k_csr_merge<double, false><<<grid, kBlock, 0, s>>>(nrows, nnz, rowptr, col, val, x, y, 1.0,
                                                        0.0, tiles, nullptr, d.carry_row,
                                                        d.carry_val, nullptr);
    CP_CUDA(cudaGetLastError());
    const int64_t fg = (tiles + kBlock - 1) / kBlock;
    k_merge_fixup<double><<<(int)(fg < cap ? fg : cap), kBlock, 0, s>>>(
        tiles, d.carry_row, d.carry_val, y, 1.0, nullptr);
    CP_CUDA(cudaGetLastError());
    return CP_OK;
  } catch (const Error& e) {
    return e.status;
  } catch (...) {
    set_error("cp_spmv_csr_merge_noalloc: unexpected internal error");
    return CP_ERR_CUDA;
  }
}
