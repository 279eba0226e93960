// CSR validation, the Table IV feature kernel, and the format conversions
// CSR -> COO / ELL / SELL-C-sigma / HYB (Sec. III-C-1: switching format needs
// new storage and a conversion kernel).  Conversions are integer work that
// copies indices and values bit for bit.
#include <algorithm>
#include <climits>
#include <cstring>

#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace cp {

void d2h_small(cp_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  CP_REQUIRE(bytes <= 4096, CP_ERR_INVALID, "staged copy too large");
  void* pin = (s == ctx->side) ? ctx->pin_side : ctx->pin_main;
  CP_CUDA(cudaMemcpyAsync(pin, src, bytes, cudaMemcpyDeviceToHost, s));
  CP_CUDA(cudaStreamSynchronize(s));
  std::memcpy(dst, pin, bytes);
}

static int grid_cap(cp_ctx* ctx, int64_t items, int block = kBlock) {
  int64_t g = (items + block - 1) / block;
  if (g > ctx->grid_stream) g = ctx->grid_stream;
  return (int)(g < 1 ? 1 : g);
}

// ================================================================== validation
enum : unsigned {
  kBadFirst = 1, kBadLast = 2, kDecreasing = 4, kRange = 8, kColRange = 16, kUnsorted = 32
};

__global__ void k_validate(int64_t n, int64_t ncols, int64_t nnz, const int32_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, unsigned* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rp[i], e = rp[i + 1];
    unsigned f = 0;
    if (i == 0 && s != 0) f |= kBadFirst;
    if (i == n - 1 && e != nnz) f |= kBadLast;
    if (e < s) f |= kDecreasing;
    if (s < 0 || e > nnz) f |= kRange;
    if (!(f & (kDecreasing | kRange))) {
      int64_t prev = -1;
      for (int64_t k = s; k < e; ++k) {
        const int64_t c = ci[k];
        if (c < 0 || c >= ncols) f |= kColRange;
        if (c <= prev) f |= kUnsorted;
        prev = c;
      }
    }
    if (f) atomicOr(err, f);
  }
}

void csr_validate(cp_ctx* ctx, cp_mat* m) {
  unsigned* d_err = dalloc<unsigned>(1);
  unsigned h_err = 0;
  try {
    CP_CUDA(cudaMemsetAsync(d_err, 0, sizeof(unsigned), ctx->main));
    CP_LAUNCH(ctx, k_validate, grid_cap(ctx, m->nrows), kBlock, 0, ctx->main, m->nrows, m->ncols,
              m->nnz, m->rowptr, m->col, d_err);
    CP_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->main));
    CP_CUDA(cudaStreamSynchronize(ctx->main));
  } catch (...) {
    dfree(d_err);
    throw;
  }
  dfree(d_err);
  CP_REQUIRE(h_err == 0, CP_ERR_INVALID,
             "invalid CSR:%s%s%s%s%s%s", (h_err & kBadFirst) ? " rowptr[0]!=0" : "",
             (h_err & kBadLast) ? " rowptr[n]!=nnz" : "",
             (h_err & kDecreasing) ? " rowptr decreasing" : "",
             (h_err & kRange) ? " rowptr out of [0,nnz]" : "",
             (h_err & kColRange) ? " column out of range" : "",
             (h_err & kUnsorted) ? " columns not strictly increasing" : "");
}

// ================================================================== features (Table IV)
struct FeatAcc {
  unsigned long long sum_r2;  // sum of squared row lengths
  unsigned long long dist;    // sum of (last col - first col)
  unsigned long long clus;    // sum of the longest consecutive-column runs
  unsigned long long ndiag;   // distinct (col - row) offsets
  unsigned maxr;              // longest row
  unsigned minr;              // shortest row (initialised to UINT_MAX)
};

constexpr int kLongRow = 64;  // rows longer than this are handled a warp at a time

// Set the bit of diagonal offset `off`.  A plain read first: structured
// matrices hit the same few offsets from every row, and an atomic per non-zero
// on those few words would serialise the whole pass.
__device__ __forceinline__ void mark_diag(unsigned* bitmap, int64_t off) {
  const unsigned bit = 1u << (off & 31);
  unsigned* w = bitmap + (off >> 5);
  if (!(*(volatile unsigned*)w & bit)) atomicOr(w, bit);
}

// A thread's last kDiagCache marked offsets.  The rows of a structured matrix
// repeat the same offsets (a stencil's rows all carry its few diagonals), so
// most marks end on a register compare and no memory request; offsets that
// miss go through mark_diag.
constexpr int kDiagCache = 16;
struct DiagCache {
  uint32_t o[kDiagCache];
  __device__ __forceinline__ DiagCache() {
#pragma unroll
    for (int k = 0; k < kDiagCache; ++k) o[k] = 0xffffffffu;
  }
  // off = col - row + nrows - 1 < 2^32 (nrows, ncols < 2^31)
  __device__ __forceinline__ void mark(unsigned* bitmap, uint32_t off) {
    bool hit = false;
#pragma unroll
    for (int k = 0; k < kDiagCache; ++k) hit |= o[k] == off;
    if (hit) return;
#pragma unroll
    for (int k = kDiagCache - 1; k > 0; --k) o[k] = o[k - 1];
    o[0] = off;
    mark_diag(bitmap, off);
  }
};

template <typename U>
__device__ __forceinline__ U warp_sum_u(U v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Pass 1: thread per row.  Lengths, sums and extremes for every row; column
// width, longest run and offsets for rows of at most kLongRow entries.
__global__ void __launch_bounds__(kBlock) k_features_rows(int64_t n, const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci,
                                                          unsigned* __restrict__ bitmap,
                                                          FeatAcc* acc) {
  unsigned long long r2 = 0, dist = 0, clus = 0;
  unsigned mx = 0, mn = UINT_MAX;
  DiagCache dc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rp[i], e = rp[i + 1];
    const unsigned len = (unsigned)(e - s);
    r2 += (unsigned long long)len * len;
    mx = max(mx, len);
    mn = min(mn, len);
    if (len == 0 || len > kLongRow) continue;
    int32_t prev = ci[s];
    dist += (unsigned long long)(ci[e - 1] - prev);
    unsigned run = 1, best = 1;
    dc.mark(bitmap, (uint32_t)((int64_t)prev - i + (n - 1)));
    for (int64_t k = s + 1; k < e; ++k) {
      const int32_t c = ci[k];
      run = (c == prev + 1) ? run + 1 : 1;
      best = max(best, run);
      dc.mark(bitmap, (uint32_t)((int64_t)c - i + (n - 1)));
      prev = c;
    }
    clus += best;
  }
  r2 = warp_sum_u(r2);
  dist = warp_sum_u(dist);
  clus = warp_sum_u(clus);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (r2) atomicAdd(&acc->sum_r2, r2);
    if (dist) atomicAdd(&acc->dist, dist);
    if (clus) atomicAdd(&acc->clus, clus);
    atomicMax(&acc->maxr, mx);
    atomicMin(&acc->minr, mn);
  }
}

// Pass 2: rows longer than kLongRow, one warp per row.  Each lane summarises a
// contiguous piece of the row (first/last column, leading and trailing runs,
// longest inner run); lane 0 folds the 32 summaries left to right.
__global__ void __launch_bounds__(kBlock) k_features_long(int64_t n, const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci,
                                                          unsigned* __restrict__ bitmap,
                                                          FeatAcc* acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long dist = 0, clus = 0;
  for (int64_t r0 = warp * 32; r0 < n; r0 += nwarps * 32) {
    const int64_t mine = r0 + lane;
    const int64_t len_mine = mine < n ? (int64_t)rp[mine + 1] - rp[mine] : 0;
    unsigned longmask = __ballot_sync(0xffffffffu, len_mine > kLongRow);
    while (longmask) {
      const int src = __ffs(longmask) - 1;
      longmask &= longmask - 1;
      const int64_t i = r0 + src;
      const int64_t s = rp[i], e = rp[i + 1], L = e - s;
      const int64_t per = (L + 31) / 32;
      const int64_t a = s + lane * per, b = min(e, a + per);
      // piece summary
      int64_t plen = b > a ? b - a : 0;
      int32_t first = 0, last = 0;
      unsigned pre = 0, suf = 0, best = 0;
      bool full = false;
      if (plen > 0) {
        first = ci[a];
        int32_t prev = first;
        unsigned run = 1;
        best = 1;
        pre = 1;
        bool in_prefix = true;
        mark_diag(bitmap, (int64_t)first - i + (n - 1));
        for (int64_t k = a + 1; k < b; ++k) {
          const int32_t c = ci[k];
          if (c == prev + 1) {
            ++run;
          } else {
            run = 1;
            in_prefix = false;
          }
          if (in_prefix) pre = run;
          best = max(best, run);
          mark_diag(bitmap, (int64_t)c - i + (n - 1));
          prev = c;
        }
        last = prev;
        suf = run;
        full = in_prefix;
      }
      // fold the 32 piece summaries in lane order (every lane takes part)
      int32_t c_last = __shfl_sync(0xffffffffu, last, 0);
      unsigned c_suf = __shfl_sync(0xffffffffu, suf, 0);
      unsigned c_best = __shfl_sync(0xffffffffu, best, 0);
      int64_t c_len = __shfl_sync(0xffffffffu, plen, 0);
      for (int j = 1; j < 32; ++j) {
        const int64_t jl = __shfl_sync(0xffffffffu, plen, j);
        const int32_t jf = __shfl_sync(0xffffffffu, first, j);
        const int32_t jlast = __shfl_sync(0xffffffffu, last, j);
        const unsigned jpre = __shfl_sync(0xffffffffu, pre, j);
        const unsigned jsuf = __shfl_sync(0xffffffffu, suf, j);
        const unsigned jbest = __shfl_sync(0xffffffffu, best, j);
        const bool jfull = __shfl_sync(0xffffffffu, (int)full, j) != 0;
        if (jl == 0) continue;
        if (c_len == 0) {
          c_last = jlast; c_suf = jsuf; c_best = jbest; c_len = jl;
          continue;
        }
        const bool joined = (jf == c_last + 1);
        if (joined) c_best = max(c_best, c_suf + jpre);
        c_best = max(c_best, jbest);
        c_suf = (jfull && joined) ? c_suf + (unsigned)jl : jsuf;
        c_last = jlast;
        c_len += jl;
      }
      if (lane == 0) {
        dist += (unsigned long long)(ci[e - 1] - ci[s]);
        clus += c_best;
      }
    }
  }
  if (lane == 0) {
    if (dist) atomicAdd(&acc->dist, dist);
    if (clus) atomicAdd(&acc->clus, clus);
  }
}

__global__ void __launch_bounds__(kBlock) k_popcount(int64_t words, const unsigned* __restrict__ bm,
                                                     FeatAcc* acc) {
  unsigned long long c = 0;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words;
       w += (int64_t)gridDim.x * blockDim.x)
    c += __popc(bm[w]);
  c = warp_sum_u(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&acc->ndiag, c);
}

__device__ double u128_to_double(unsigned long long hi, unsigned long long lo) {
  return (double)hi * 18446744073709551616.0 + (double)lo;
}

// One thread: the 15 features from the exact integer sums, fixed formulas.
__global__ void k_features_final(int64_t n, int64_t ncols, int64_t nnz, const FeatAcc* acc,
                                 double* f) {
  const double dn = (double)n, dnnz = (double)nnz;
  const double mean = dnnz / dn;
  // population variance = (n * sum r^2 - nnz^2) / n^2, numerator exact in 128 bits
  const unsigned __int128 a = (unsigned __int128)(unsigned long long)n * acc->sum_r2;
  const unsigned __int128 b = (unsigned __int128)(unsigned long long)nnz * (unsigned long long)nnz;
  const unsigned __int128 num = a - b;
  const double var = u128_to_double((unsigned long long)(num >> 64), (unsigned long long)num) /
                     (dn * dn);
  const double sd = sqrt(var);
  const double mx = (double)acc->maxr, mn = (double)acc->minr, nd = (double)acc->ndiag;
  f[0] = dn;
  f[1] = (double)ncols;
  f[2] = dnnz;
  f[3] = dnnz / (dn * (double)ncols);
  f[4] = mean;
  f[5] = sd;
  f[6] = mean != 0.0 ? sd / mean : 0.0;
  f[7] = mx;
  f[8] = mn;
  f[9] = mx - mean;
  f[10] = (double)acc->dist / dn;
  f[11] = (double)acc->clus / dn;
  f[12] = nnz > 0 ? dn * mx / dnnz : 0.0;
  f[13] = nd;
  f[14] = nnz > 0 ? dn * nd / dnnz : 0.0;
}

void compute_features(cp_ctx* ctx, cp_mat* m, cudaStream_t s, double* out15) {
  std::lock_guard<std::mutex> lock(m->feat_mu);
  if (m->has_features) {
    std::memcpy(out15, m->features, sizeof(m->features));
    return;
  }
  const int64_t n = m->nrows;
  const int64_t words = (n + m->ncols - 1 + 31) / 32;
  void* scratch = nullptr;
  unsigned* bm = nullptr;  // kept for the DIA conversion (m->diag_bm)
  const size_t bytes = sizeof(FeatAcc) + 15 * sizeof(double);
  trace("features: start n=%lld", (long long)n);
  CP_CUDA(cudaMallocAsync(&scratch, bytes, s));
  trace("features: scratch allocated");
  FeatAcc* acc = static_cast<FeatAcc*>(scratch);
  double* f = reinterpret_cast<double*>(static_cast<char*>(scratch) + sizeof(FeatAcc));
  try {
    bm = dalloc_async<unsigned>(words, s);
    CP_CUDA(cudaMemsetAsync(scratch, 0, bytes, s));
    CP_CUDA(cudaMemsetAsync(bm, 0, words * sizeof(unsigned), s));
    CP_CUDA(cudaMemsetAsync(&acc->minr, 0xff, sizeof(unsigned), s));
    const int g = grid_cap(ctx, n);
    CP_LAUNCH(ctx, k_features_rows, g, kBlock, 0, s, n, m->rowptr, m->col, bm, acc);
    CP_LAUNCH(ctx, k_features_long, grid_cap(ctx, n), kBlock, 0, s, n, m->rowptr, m->col, bm, acc);
    CP_LAUNCH(ctx, k_popcount, grid_cap(ctx, words), kBlock, 0, s, words, bm, acc);
    CP_LAUNCH(ctx, k_features_final, 1, 1, 0, s, n, m->ncols, m->nnz, acc, f);
    trace("features: kernels queued");
    d2h_small(ctx, m->features, f, 15 * sizeof(double), s);  // waits for the kernels
    trace("features: done");
    CP_CUDA(cudaFreeAsync(scratch, s));
  } catch (...) {
    cudaFreeAsync(scratch, s);
    dfree_async(bm, s);
    throw;
  }
  if (unsigned* old = m->diag_bm.exchange(bm)) dfree_async(old, s);
  m->has_features = true;
  std::memcpy(out15, m->features, sizeof(m->features));
}

// ================================================================== scan
constexpr int kScanItems = 4;
constexpr int kScanTile = kBlock * kScanItems;

// Exclusive scan of one tile per block; block totals to sums[] (if non-null).
__global__ void __launch_bounds__(kBlock) k_scan_tile(const int64_t* __restrict__ in,
                                                      int64_t* __restrict__ out, int64_t n,
                                                      int64_t* __restrict__ sums) {
  __shared__ int64_t warp_tot[kBlock / 32];
  const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t t = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < n ? in[base + j] : 0;
    t += v[j];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t up = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += up;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  int64_t woff = 0;
  for (int w = 0; w < warp; ++w) woff += warp_tot[w];
  int64_t run = woff + inc - t;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
  if (sums && threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
  const int64_t i = blockIdx.x * (int64_t)kScanTile;
  const int64_t off = offs[blockIdx.x];
  for (int j = threadIdx.x; j < kScanTile && i + j < n; j += blockDim.x) out[i + j] += off;
}

__global__ void k_scan_total(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n) {
  out[n] = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

void exclusive_scan_i64(cp_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles <= 1) {
    CP_LAUNCH(ctx, k_scan_tile, 1, kBlock, 0, s, in, out, n, (int64_t*)nullptr);
  } else {
    int64_t* sums = nullptr;
    CP_CUDA(cudaMallocAsync(&sums, sizeof(int64_t) * (2 * tiles + 1), s));
    int64_t* offs = sums + tiles;
    CP_LAUNCH(ctx, k_scan_tile, (int)tiles, kBlock, 0, s, in, out, n, sums);
    exclusive_scan_i64(ctx, sums, offs, tiles, s);
    CP_LAUNCH(ctx, k_scan_add, (int)tiles, kBlock, 0, s, out, n, offs);
    CP_CUDA(cudaFreeAsync(sums, s));
  }
  CP_LAUNCH(ctx, k_scan_total, 1, 1, 0, s, in, out, n);
}

// ================================================================== conversions
__global__ void k_coo_rows(int64_t n, const int32_t* __restrict__ rp, int32_t* __restrict__ row) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) row[k] = (int32_t)i;
}

// ELL part of width K for rows [0, ld): the first min(len, K) entries of row i.
__global__ void __launch_bounds__(kBlock) k_ell_fill(int64_t n, int64_t ld, int64_t K,
                                                     const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ ci,
                                                     const double* __restrict__ v,
                                                     int32_t* __restrict__ ec,
                                                     double* __restrict__ ev) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ld;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i < n ? rp[i] : 0;
    const int64_t len = i < n ? rp[i + 1] - s : 0;
    for (int64_t k = 0; k < K; ++k) {
      if (k < len) {
        ec[k * ld + i] = ci[s + k];
        ev[k * ld + i] = v[s + k];
      } else {
        ec[k * ld + i] = -1;
        ev[k * ld + i] = 0.0;
      }
    }
  }
}

__global__ void k_hyb_counts(int64_t n, int64_t K, const int32_t* __restrict__ rp,
                             int64_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t len = rp[i + 1] - rp[i];
    cnt[i] = len > K ? len - K : 0;
  }
}

__global__ void k_hyb_coo_fill(int64_t n, int64_t K, const int32_t* __restrict__ rp,
                               const int32_t* __restrict__ ci, const double* __restrict__ v,
                               const int64_t* __restrict__ off, int32_t* __restrict__ cr,
                               int32_t* __restrict__ cc, double* __restrict__ cv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rp[i], e = rp[i + 1];
    int64_t o = off[i];
    for (int64_t k = s + K; k < e; ++k, ++o) {
      cr[o] = (int32_t)i;
      cc[o] = ci[k];
      cv[o] = v[k];
    }
  }
}

__global__ void k_iota(int64_t n, int32_t* p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

// One block per window of sigma rows: bitonic sort of the keys
// (INT32_MAX - length, position in window) ascending, i.e. longest first with
// ties in original order.  Keys are padded to the next power of two.
__global__ void __launch_bounds__(1024) k_sell_sort(int64_t n, int64_t sigma, int pow2,
                                                    const int32_t* __restrict__ rp,
                                                    int32_t* __restrict__ perm) {
  extern __shared__ unsigned long long keys[];
  const int64_t w0 = blockIdx.x * sigma;
  const int64_t wn = (w0 + sigma < n ? w0 + sigma : n) - w0;
  for (int j = threadIdx.x; j < pow2; j += blockDim.x) {
    if (j < wn) {
      const int64_t len = rp[w0 + j + 1] - rp[w0 + j];
      keys[j] = ((unsigned long long)(0x7fffffffLL - len) << 32) | (unsigned)j;
    } else {
      keys[j] = ~0ull;
    }
  }
  __syncthreads();
  for (int size = 2; size <= pow2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int j = threadIdx.x; j < pow2; j += blockDim.x) {
        const int p = j ^ stride;
        if (p > j) {
          const bool up = (j & size) == 0;
          const unsigned long long a = keys[j], b = keys[p];
          if ((a > b) == up) {
            keys[j] = b;
            keys[p] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j < wn; j += blockDim.x)
    perm[w0 + j] = (int32_t)(w0 + (keys[j] & 0xffffffffu));
}

// Warp per chunk: width = longest row in the chunk; count = C * width.
__global__ void __launch_bounds__(kBlock) k_sell_widths(int64_t n, int64_t nchunks,
                                                        const int32_t* __restrict__ rp,
                                                        const int32_t* __restrict__ perm,
                                                        int32_t* __restrict__ clen,
                                                        int64_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < nchunks; c += nwarps) {
    const int64_t s = c * 32 + lane;
    int len = 0;
    if (s < n) {
      const int32_t r = perm[s];
      len = rp[r + 1] - rp[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if (lane == 0) {
      clen[c] = len;
      cnt[c] = 32ll * len;
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_sell_fill(int64_t n, int64_t nchunks,
                                                      const int32_t* __restrict__ rp,
                                                      const int32_t* __restrict__ ci,
                                                      const double* __restrict__ v,
                                                      const int32_t* __restrict__ perm,
                                                      const int32_t* __restrict__ clen,
                                                      const int64_t* __restrict__ cptr,
                                                      int32_t* __restrict__ sc,
                                                      double* __restrict__ sv) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = warp; c < nchunks; c += nwarps) {
    const int64_t slot = c * 32 + lane;
    int64_t s = 0, len = 0;
    if (slot < n) {
      const int32_t r = perm[slot];
      s = rp[r];
      len = rp[r + 1] - s;
    }
    const int64_t base = cptr[c] + lane;
    const int w = clen[c];
    for (int k = 0; k < w; ++k) {
      if (k < len) {
        sc[base + (int64_t)k * 32] = ci[s + k];
        sv[base + (int64_t)k * 32] = v[s + k];
      } else {
        sc[base + (int64_t)k * 32] = -1;
        sv[base + (int64_t)k * 32] = 0.0;
      }
    }
  }
}

__global__ void k_cast_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __double2float_rn(a[i]);
}

// DIA conversion: mark the offsets present, compact them in ascending order
// (word popcounts -> exclusive scan -> each word writes its bits), then fill
// every slot of every row once.
__global__ void __launch_bounds__(kBlock) k_dia_mark(int64_t n, const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ ci,
                                                     unsigned* __restrict__ bm) {
  DiagCache dc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
      dc.mark(bm, (uint32_t)((int64_t)ci[k] - i + (n - 1)));
}

__global__ void k_dia_wordcount(int64_t words, const unsigned* __restrict__ bm,
                                int64_t* __restrict__ cnt) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words;
       w += (int64_t)gridDim.x * blockDim.x)
    cnt[w] = __popc(bm[w]);
}

__global__ void k_dia_compact(int64_t n, int64_t words, const unsigned* __restrict__ bm,
                              const int64_t* __restrict__ pos, int32_t* __restrict__ offs,
                              int64_t cap) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words;
       w += (int64_t)gridDim.x * blockDim.x) {
    unsigned bits = bm[w];
    int64_t q = pos[w];
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      const int64_t o = w * 32 + b;  // offset + (n - 1)
      if (q < cap) offs[q] = (int32_t)(o - (n - 1));
      ++q;
    }
  }
}

// A thread per row walks the row's entries (ascending columns) and the
// diagonals (ascending offsets, in shared memory) together and writes every
// slot of the row once: the entry on that diagonal, or zero.  Every entry lies
// on a diagonal that was marked, so the walk takes each entry in turn; no slot
// is written twice (no zero fill of the whole array first) and no offset ->
// diagonal table is read per entry.
__global__ void __launch_bounds__(kBlock) k_dia_fill(int64_t n, int ndiag,
                                                     const int32_t* __restrict__ offs,
                                                     const int32_t* __restrict__ rp,
                                                     const int32_t* __restrict__ ci,
                                                     const double* __restrict__ v,
                                                     double* __restrict__ data) {
  __shared__ int32_t so[kDiaMax];
  for (int d = threadIdx.x; d < ndiag; d += blockDim.x) so[d] = offs[d];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = rp[i];
    const int64_t e = rp[i + 1];
    int64_t c = k < e ? (int64_t)ci[k] : INT64_MAX;  // the next entry's column
    for (int d = 0; d < ndiag; ++d) {
      double val = 0.0;
      if (c == i + so[d]) {
        val = v[k];
        ++k;
        c = k < e ? (int64_t)ci[k] : INT64_MAX;
      }
      data[(int64_t)d * n + i] = val;
    }
  }
}

// ------------------------------------------------------------------ host side
void config_check(const cp_config& c) {
  CP_REQUIRE(c.fmt >= 0 && c.fmt < CP_NUM_FMT, CP_ERR_UNSUPPORTED, "unknown format %d", c.fmt);
  if (c.fmt == CP_FMT_CSR) {
    CP_REQUIRE(c.algo >= 0 && c.algo < CP_NUM_ALGO, CP_ERR_UNSUPPORTED, "unknown CSR algorithm %d",
               c.algo);
    if (c.algo == CP_ALGO_VECTOR)
      CP_REQUIRE(c.tpv == 2 || c.tpv == 4 || c.tpv == 8 || c.tpv == 16 || c.tpv == 32,
                 CP_ERR_UNSUPPORTED, "TpV must be 2, 4, 8, 16 or 32 (got %d)", c.tpv);
  }
  if (c.fmt == CP_FMT_SELL) {
    CP_REQUIRE(c.sell_c == 32, CP_ERR_UNSUPPORTED, "SELL chunk height must be 32 (got %d)",
               c.sell_c);
    CP_REQUIRE(c.sell_sigma == 1 || (c.sell_sigma > 0 && c.sell_sigma % 32 == 0 &&
                                     c.sell_sigma <= 8192),
               CP_ERR_UNSUPPORTED, "SELL sigma must be 1 or a multiple of 32 up to 8192 (got %d)",
               c.sell_sigma);
  }
  if (c.fmt == CP_FMT_HYB) CP_REQUIRE(c.hyb_k >= 0, CP_ERR_UNSUPPORTED, "HYB K must be >= 0");
}

bool config_equal(const cp_config& a, const cp_config& b) {
  if (a.fmt != b.fmt) return false;
  switch (a.fmt) {
    case CP_FMT_CSR:
      return a.algo == b.algo && (a.algo != CP_ALGO_VECTOR || a.tpv == b.tpv);
    case CP_FMT_SELL:
      return a.sell_sigma == b.sell_sigma;
    case CP_FMT_HYB:
      return a.hyb_k == b.hyb_k;
    default:
      return true;
  }
}

// Rows by length for HYB's width rule: lengths 0 .. kLenBins - 2, longer rows
// in the last bin.
constexpr int kLenBins = 1024;
__global__ void k_row_length_hist(int64_t n, const int32_t* __restrict__ rp,
                                  unsigned* __restrict__ hist) {
  __shared__ unsigned h[kLenBins];
  for (int i = threadIdx.x; i < kLenBins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t len = (int64_t)rp[i + 1] - rp[i];
    atomicAdd(&h[len < kLenBins - 1 ? len : kLenBins - 1], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kLenBins; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// HYB's ELL width K (Sec. III-B-2 lists it among the format's parameters; the
// paper fixes no default).  hyb_k > 0 gives it.  Otherwise K is the smallest
// width (at least 1) that at most a quarter of the rows exceed, the 75th
// percentile of the row lengths: one more slot a row costs n ELL slots and
// saves one COO entry per longer row, and on this GPU a COO entry costs about
// four ELL slots (a fit of HYB SpMV times over K on a power-law matrix), so the
// total stops falling where a quarter of the rows are longer.  If that
// percentile is past the histogram (rows of 1,023 entries or more),
// ceil(mean row length).  Found once per matrix.
int64_t hyb_width(cp_ctx* ctx, cp_mat* m, const cp_config& c, cudaStream_t s) {
  if (c.hyb_k > 0) return c.hyb_k;
  if (m->hyb_auto_k > 0) return m->hyb_auto_k;
  unsigned* d = dalloc_async<unsigned>(kLenBins, s);
  std::vector<unsigned> h(kLenBins);
  try {
    CP_CUDA(cudaMemsetAsync(d, 0, kLenBins * sizeof(unsigned), s));
    CP_LAUNCH(ctx, k_row_length_hist, grid_cap(ctx, m->nrows), kBlock, 0, s, m->nrows,
              m->rowptr, d);
    static_assert(kLenBins * sizeof(unsigned) <= 4096, "one staged copy");
    d2h_small(ctx, h.data(), d, kLenBins * sizeof(unsigned), s);
  } catch (...) {
    dfree_async(d, s);
    throw;
  }
  dfree_async(d, s);
  int64_t K = 0, over = m->nrows - (int64_t)h[0];  // rows longer than K
  while (K < kLenBins - 2 && (K < 1 || 4 * over > m->nrows)) {
    ++K;
    over -= h[K];
  }
  if (4 * over > m->nrows) {  // the percentile is in the last bin
    K = (m->nnz + m->nrows - 1) / m->nrows;
    if (K < 1) K = 1;
  }
  m->hyb_auto_k = K;
  return K;
}

static void free_ell(EllPart& e) {
  dfree(e.col);
  dfree(e.val);
  dfree(e.val32);
  e = EllPart{};
}
static void free_coo(CooPart& c) {
  dfree(c.row);
  if (c.owns_colval) {
    dfree(c.col);
    dfree(c.val);
  }
  dfree(c.val32);
  c = CooPart{};
}
static void free_sell(SellPart& s) {
  dfree(s.perm);
  dfree(s.chunk_len);
  dfree(s.chunk_ptr);
  dfree(s.col);
  dfree(s.val);
  dfree(s.val32);
  s = SellPart{};
}

static void free_dia(DiaPart& d);

void free_formats(cp_mat* m) {
  free_coo(m->coo);
  free_ell(m->ell);
  free_sell(m->sell);
  free_ell(m->hyb_ell);
  free_coo(m->hyb_coo);
  free_dia(m->dia);
  dfree(m->diag_bm.exchange(nullptr));
  m->has_coo = m->has_ell = m->has_sell = m->has_hyb = m->has_dia = false;
  dfree(m->merge_carry_row);
  dfree(m->merge_carry_val);
  dfree(m->merge_start);
  m->merge_carry_row = nullptr;
  m->merge_carry_val = nullptr;
  m->merge_start = nullptr;
  m->merge_tiles = 0;
  if (m->merge_err) m->ctx->mapped.give(m->merge_err);
  m->merge_err = nullptr;
  m->merge_err_dev = nullptr;
  dfree(m->val32);
  m->val32 = nullptr;
}

static void check_budget(cp_ctx* ctx, int64_t bytes, const char* what) {
  CP_REQUIRE(bytes <= ctx->format_budget, CP_ERR_FOOTPRINT,
             "%s needs %lld bytes, above the format budget of %lld bytes", what, (long long)bytes,
             (long long)ctx->format_budget);
}

static void convert_ell(cp_ctx* ctx, cp_mat* m, cudaStream_t s) {
  double f[15];
  compute_features(ctx, m, s, f);
  EllPart e;
  e.K = (int64_t)f[7];
  e.ld = (m->nrows + 31) / 32 * 32;
  check_budget(ctx, e.K * e.ld * 12, "ELL");
  try {
    e.col = dalloc_async<int32_t>(e.K * e.ld, s);
    e.val = dalloc_async<double>(e.K * e.ld, s);
    CP_LAUNCH(ctx, k_ell_fill, grid_cap(ctx, e.ld), kBlock, 0, s, m->nrows, e.ld, e.K, m->rowptr,
              m->col, m->val, e.col, e.val);
    CP_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    free_ell(e);
    throw;
  }
  m->ell = e;
  m->has_ell = true;
}

static void convert_coo(cp_ctx* ctx, cp_mat* m, cudaStream_t s) {
  CooPart c;
  c.n = m->nnz;
  c.col = m->col;
  c.val = m->val;
  c.owns_colval = false;
  try {
    c.row = dalloc_async<int32_t>(m->nnz, s);
    CP_LAUNCH(ctx, k_coo_rows, grid_cap(ctx, m->nrows), kBlock, 0, s, m->nrows, m->rowptr, c.row);
    CP_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    free_coo(c);
    throw;
  }
  m->coo = c;
  m->has_coo = true;
}

static void convert_sell(cp_ctx* ctx, cp_mat* m, int64_t sigma, cudaStream_t s) {
  SellPart p;
  p.C = 32;
  p.sigma = sigma;
  p.nchunks = (m->nrows + 31) / 32;
  int64_t* cnt = nullptr;
  try {
    p.perm = dalloc_async<int32_t>(m->nrows, s);
    p.chunk_len = dalloc_async<int32_t>(p.nchunks, s);
    p.chunk_ptr = dalloc_async<int64_t>(p.nchunks + 1, s);
    cnt = dalloc_async<int64_t>(p.nchunks, s);
    if (sigma == 1) {
      CP_LAUNCH(ctx, k_iota, grid_cap(ctx, m->nrows), kBlock, 0, s, m->nrows, p.perm);
    } else {
      int pow2 = 1;
      while (pow2 < sigma) pow2 <<= 1;
      const int smem = pow2 * (int)sizeof(unsigned long long);
      CP_CUDA(cudaFuncSetAttribute(k_sell_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      const int64_t windows = (m->nrows + sigma - 1) / sigma;
      CP_LAUNCH(ctx, k_sell_sort, (int)windows, 1024, smem, s, m->nrows, sigma, pow2, m->rowptr,
                p.perm);
    }
    CP_LAUNCH(ctx, k_sell_widths, grid_cap(ctx, p.nchunks * 32), kBlock, 0, s, m->nrows,
              p.nchunks, m->rowptr, p.perm, p.chunk_len, cnt);
    exclusive_scan_i64(ctx, cnt, p.chunk_ptr, p.nchunks, s);
    dfree_async(cnt, s);
    cnt = nullptr;
    d2h_small(ctx, &p.slots, p.chunk_ptr + p.nchunks, sizeof(int64_t), s);
    check_budget(ctx, p.slots * 12, "SELL-C-sigma");
    p.col = dalloc_async<int32_t>(p.slots, s);
    p.val = dalloc_async<double>(p.slots, s);
    CP_LAUNCH(ctx, k_sell_fill, grid_cap(ctx, p.nchunks * 32), kBlock, 0, s, m->nrows, p.nchunks,
              m->rowptr, m->col, m->val, p.perm, p.chunk_len, p.chunk_ptr, p.col, p.val);
    CP_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    dfree_async(cnt, s);
    free_sell(p);
    throw;
  }
  free_sell(m->sell);
  m->sell = p;
  m->has_sell = true;
}

static void convert_hyb(cp_ctx* ctx, cp_mat* m, int64_t K, cudaStream_t s) {
  EllPart e;
  CooPart c;
  int64_t* cnt = nullptr;
  int64_t* off = nullptr;
  e.K = K;
  e.ld = (m->nrows + 31) / 32 * 32;
  check_budget(ctx, e.K * e.ld * 12, "HYB ELL part");
  try {
    e.col = dalloc_async<int32_t>(e.K * e.ld, s);
    e.val = dalloc_async<double>(e.K * e.ld, s);
    CP_LAUNCH(ctx, k_ell_fill, grid_cap(ctx, e.ld), kBlock, 0, s, m->nrows, e.ld, e.K, m->rowptr,
              m->col, m->val, e.col, e.val);
    cnt = dalloc_async<int64_t>(m->nrows, s);
    off = dalloc_async<int64_t>(m->nrows + 1, s);
    CP_LAUNCH(ctx, k_hyb_counts, grid_cap(ctx, m->nrows), kBlock, 0, s, m->nrows, K, m->rowptr,
              cnt);
    exclusive_scan_i64(ctx, cnt, off, m->nrows, s);
    d2h_small(ctx, &c.n, off + m->nrows, sizeof(int64_t), s);
    c.owns_colval = true;
    c.row = dalloc_async<int32_t>(c.n, s);
    c.col = dalloc_async<int32_t>(c.n, s);
    c.val = dalloc_async<double>(c.n, s);
    if (c.n > 0)
      CP_LAUNCH(ctx, k_hyb_coo_fill, grid_cap(ctx, m->nrows), kBlock, 0, s, m->nrows, K,
                m->rowptr, m->col, m->val, off, c.row, c.col, c.val);
    CP_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    dfree_async(cnt, s);
    dfree_async(off, s);
    free_ell(e);
    free_coo(c);
    throw;
  }
  dfree_async(cnt, s);
  dfree_async(off, s);
  free_ell(m->hyb_ell);
  free_coo(m->hyb_coo);
  m->hyb_ell = e;
  m->hyb_coo = c;
  m->has_hyb = true;
}

static void free_dia(DiaPart& d) {
  dfree(d.offs);
  dfree(d.val);
  dfree(d.val32);
  d = DiaPart{};
}

static void convert_dia(cp_ctx* ctx, cp_mat* m, cudaStream_t s) {
  const int64_t n = m->nrows;
  const int64_t span = n + m->ncols - 1;
  const int64_t words = (span + 31) / 32;
  DiaPart d;
  // the offsets present: the feature pass's bitmap when it ran (complete once
  // published), else marked here
  unsigned* const have = m->diag_bm.load();
  unsigned* bm = have;
  int64_t *cnt = nullptr, *pos = nullptr;
  try {
    cnt = dalloc_async<int64_t>(words, s);
    pos = dalloc_async<int64_t>(words + 1, s);
    d.offs = dalloc_async<int32_t>(kDiaMax, s);
    if (!have) {
      bm = dalloc_async<unsigned>(words, s);
      CP_CUDA(cudaMemsetAsync(bm, 0, words * sizeof(unsigned), s));
      CP_LAUNCH(ctx, k_dia_mark, grid_cap(ctx, n), kBlock, 0, s, n, m->rowptr, m->col, bm);
    }
    CP_LAUNCH(ctx, k_dia_wordcount, grid_cap(ctx, words), kBlock, 0, s, words, bm, cnt);
    exclusive_scan_i64(ctx, cnt, pos, words, s);
    CP_LAUNCH(ctx, k_dia_compact, grid_cap(ctx, words), kBlock, 0, s, n, words, bm, pos, d.offs,
              (int64_t)kDiaMax);
    d2h_small(ctx, &d.ndiag, pos + words, sizeof(int64_t), s);
    CP_REQUIRE(d.ndiag <= kDiaMax, CP_ERR_FOOTPRINT,
               "DIA needs %lld diagonals, more than the %d it accepts", (long long)d.ndiag,
               kDiaMax);
    check_budget(ctx, d.ndiag * n * 8, "DIA");
    d.val = dalloc_async<double>(d.ndiag * n, s);
    CP_LAUNCH(ctx, k_dia_fill, grid_cap(ctx, n), kBlock, 0, s, n, (int)d.ndiag, d.offs,
              m->rowptr, m->col, m->val, d.val);
    CP_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    if (!have) dfree_async(bm, s);
    dfree_async(cnt, s);
    dfree_async(pos, s);
    free_dia(d);
    throw;
  }
  if (!have) dfree_async(bm, s);
  dfree_async(cnt, s);
  dfree_async(pos, s);
  m->dia = d;
  m->has_dia = true;
}

// Merge-path set-up, once per matrix: the per-tile carries and the tile start
// points (the matrix is fixed, so the diagonal searches are not repeated in
// every SpMV).
static void prepare_merge(cp_ctx* ctx, cp_mat* m, cudaStream_t s) {
  const int64_t tiles = (m->nrows + m->nnz + kMergeWarpTile - 1) / kMergeWarpTile;
  if (m->merge_tiles == tiles && m->merge_carry_row) return;
  dfree(m->merge_carry_row);
  dfree(m->merge_carry_val);
  dfree(m->merge_start);
  m->merge_carry_row = dalloc_async<int32_t>(tiles, s);
  m->merge_carry_val = dalloc_async<double>(tiles, s);
  m->merge_start = dalloc_async<int32_t>(tiles + 1, s);
  m->merge_tiles = tiles;
  if (!m->merge_err) {
    m->merge_err = static_cast<int*>(ctx->mapped.take());
    CP_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&m->merge_err_dev), m->merge_err,
                                     0));
  }
  merge_partition(ctx, m, s);
  CP_CUDA(cudaStreamSynchronize(s));
}

void ensure_format(cp_ctx* ctx, cp_mat* m, const cp_config& cfg, cudaStream_t s) {
  config_check(cfg);
  std::lock_guard<std::mutex> lock(m->mu);
  switch (cfg.fmt) {
    case CP_FMT_CSR:
      if (cfg.algo == CP_ALGO_MERGE) prepare_merge(ctx, m, s);
      break;
    case CP_FMT_COO:
      if (!m->has_coo) convert_coo(ctx, m, s);
      break;
    case CP_FMT_ELL:
      if (!m->has_ell) convert_ell(ctx, m, s);
      break;
    case CP_FMT_SELL:
      if (!m->has_sell || m->sell.sigma != cfg.sell_sigma) convert_sell(ctx, m, cfg.sell_sigma, s);
      break;
    case CP_FMT_HYB: {
      const int64_t K = hyb_width(ctx, m, cfg, s);
      if (!m->has_hyb || m->hyb_ell.K != K) convert_hyb(ctx, m, K, s);
      break;
    }
    case CP_FMT_DIA:
      if (!m->has_dia) convert_dia(ctx, m, s);
      break;
  }
}

static float* cast_copy(cp_ctx* ctx, const double* src, int64_t n, cudaStream_t s) {
  float* d = dalloc_async<float>(n, s);
  if (n > 0) CP_LAUNCH(ctx, k_cast_f32, grid_cap(ctx, n), kBlock, 0, s, n, src, d);
  return d;
}

void ensure_val32(cp_ctx* ctx, cp_mat* m, const cp_config& cfg, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(m->mu);
  switch (cfg.fmt) {
    case CP_FMT_CSR:
    case CP_FMT_COO:
      if (!m->val32) m->val32 = cast_copy(ctx, m->val, m->nnz, s);
      break;
    case CP_FMT_ELL:
      if (!m->ell.val32) m->ell.val32 = cast_copy(ctx, m->ell.val, m->ell.K * m->ell.ld, s);
      break;
    case CP_FMT_SELL:
      if (!m->sell.val32) m->sell.val32 = cast_copy(ctx, m->sell.val, m->sell.slots, s);
      break;
    case CP_FMT_HYB:
      if (!m->hyb_ell.val32)
        m->hyb_ell.val32 = cast_copy(ctx, m->hyb_ell.val, m->hyb_ell.K * m->hyb_ell.ld, s);
      if (!m->hyb_coo.val32) m->hyb_coo.val32 = cast_copy(ctx, m->hyb_coo.val, m->hyb_coo.n, s);
      break;
    case CP_FMT_DIA:
      if (!m->dia.val32) m->dia.val32 = cast_copy(ctx, m->dia.val, m->dia.ndiag * m->nrows, s);
      break;
  }
  CP_CUDA(cudaStreamSynchronize(s));
}

void format_dims(cp_mat* m, const cp_config& cfg, int64_t dims[4]) {
  dims[0] = dims[1] = dims[2] = dims[3] = 0;
  switch (cfg.fmt) {
    case CP_FMT_ELL:
      dims[0] = m->ell.K;
      dims[1] = m->ell.ld;
      break;
    case CP_FMT_SELL:
      dims[0] = m->sell.nchunks;
      dims[1] = m->sell.slots;
      dims[2] = m->sell.C;
      dims[3] = m->sell.sigma;
      break;
    case CP_FMT_HYB:
      dims[0] = m->hyb_ell.K;
      dims[1] = m->hyb_ell.ld;
      dims[2] = m->hyb_coo.n;
      break;
    case CP_FMT_COO:
      dims[0] = m->nnz;
      break;
    case CP_FMT_DIA:
      dims[0] = m->dia.ndiag;
      dims[1] = m->nrows;
      break;
    default:
      break;
  }
}

void format_export(cp_mat* m, const cp_config& cfg, int id, void* dst, int64_t cap,
                   int64_t* bytes, cudaStream_t s) {
  const void* src = nullptr;
  int64_t nb = 0;
  switch (id) {
    case CP_ARR_COO_ROW: src = m->coo.row; nb = m->nnz * 4; break;
    case CP_ARR_ELL_COL: src = m->ell.col; nb = m->ell.K * m->ell.ld * 4; break;
    case CP_ARR_ELL_VAL: src = m->ell.val; nb = m->ell.K * m->ell.ld * 8; break;
    case CP_ARR_SELL_PERM: src = m->sell.perm; nb = m->nrows * 4; break;
    case CP_ARR_SELL_CHUNK_LEN: src = m->sell.chunk_len; nb = m->sell.nchunks * 4; break;
    case CP_ARR_SELL_CHUNK_PTR: src = m->sell.chunk_ptr; nb = (m->sell.nchunks + 1) * 8; break;
    case CP_ARR_SELL_COL: src = m->sell.col; nb = m->sell.slots * 4; break;
    case CP_ARR_SELL_VAL: src = m->sell.val; nb = m->sell.slots * 8; break;
    case CP_ARR_HYB_ELL_COL: src = m->hyb_ell.col; nb = m->hyb_ell.K * m->hyb_ell.ld * 4; break;
    case CP_ARR_HYB_ELL_VAL: src = m->hyb_ell.val; nb = m->hyb_ell.K * m->hyb_ell.ld * 8; break;
    case CP_ARR_HYB_COO_ROW: src = m->hyb_coo.row; nb = m->hyb_coo.n * 4; break;
    case CP_ARR_HYB_COO_COL: src = m->hyb_coo.col; nb = m->hyb_coo.n * 4; break;
    case CP_ARR_HYB_COO_VAL: src = m->hyb_coo.val; nb = m->hyb_coo.n * 8; break;
    case CP_ARR_DIA_OFFSETS: src = m->dia.offs; nb = m->dia.ndiag * 4; break;
    case CP_ARR_DIA_VAL: src = m->dia.val; nb = m->dia.ndiag * m->nrows * 8; break;
    default: CP_REQUIRE(false, CP_ERR_INVALID, "unknown array id %d", id);
  }
  (void)cfg;
  *bytes = nb;
  CP_REQUIRE(nb <= cap, CP_ERR_INVALID, "export needs %lld bytes, capacity %lld", (long long)nb,
             (long long)cap);
  if (nb > 0) {
    CP_CUDA(cudaMemcpyAsync(dst, src, nb, cudaMemcpyDeviceToHost, s));
    CP_CUDA(cudaStreamSynchronize(s));
  }
}

}  // namespace cp
