// Row loops of the row-parallel SpMV formats (CSR-scalar, CSR-vector, ELL,
// SELL-C-sigma, DIA).  Each walks its rows grid-stride from the caller's
// thread (or warp) index, writes y = A x (or alpha A x + beta y) and returns the
// thread's share of sum_i y_i * dotv_i when DOT is set.  The SpMV kernels of
// spmv.cu wrap them one launch each; the persistent CG kernel runs them as the
// SpMV phase of every iteration with COH set, so the x and dot vectors (which
// that kernel rewrites every iteration) are read through L2, never from a
// possibly stale L1 or read-only-cache line.
#pragma once

#include "common.cuh"
#include "internal.cuh"

namespace cp {

// y_i <- s (solver form) or alpha s + beta y_i (general form; y not read when beta = 0)
template <typename T, bool GEN>
__device__ __forceinline__ void store_row(T* y, int64_t i, T s, T alpha, T beta) {
  if (GEN) {
    T r = alpha * s;
    if (beta != T(0)) r = fma(beta, y[i], r);
    y[i] = r;
  } else {
    y[i] = s;
  }
}

// ------------------------------------------------------------------ CSR scalar
// One thread per row; entries in chunks of 4 so the 8 index / value loads are
// independent, then 4 gathers.
template <typename T, bool GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T csr_scalar_rows(int64_t n, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci,
                                             const T* __restrict__ v, const T* __restrict__ x,
                                             T* __restrict__ y, T alpha, T beta,
                                             const T* __restrict__ dotv, int64_t tid,
                                             int64_t stride) {
  T acc = 0;
  for (int64_t i = tid; i < n; i += stride) {
    const int s = rp[i], e = rp[i + 1];
    T sum = 0;
    for (int k0 = s; k0 < e; k0 += 4) {
      int32_t c[4];
      T w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = k0 + u < e;
        c[u] = in ? ld_stream(ci + k0 + u) : 0;
        w[u] = in ? ld_stream(v + k0 + u) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k0 + u < e) sum = fma(w[u], ld_x<COH>(x + c[u]), sum);
    }
    store_row<T, GEN>(y, i, sum, alpha, beta);
    if (DOT) acc = fma(sum, COH ? ld_cg(dotv + i) : dotv[i], acc);
  }
  return acc;
}

// ------------------------------------------------------------------ CSR vector
// TPV lanes per row; the warp walks its rows in lock step so the shuffles of
// the row reduction always see the full warp.  warp / nwarps: global warp index
// and count.
template <typename T, int TPV, bool GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T csr_vector_rows(int64_t n, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci,
                                             const T* __restrict__ v, const T* __restrict__ x,
                                             T* __restrict__ y, T alpha, T beta,
                                             const T* __restrict__ dotv, int64_t warp,
                                             int64_t nwarps) {
  constexpr int RPW = 32 / TPV;  // rows per warp step
  const int lane = threadIdx.x & 31;
  const int sub = lane % TPV;
  T acc = 0;
  for (int64_t r0 = warp * RPW; r0 < n; r0 += nwarps * RPW) {
    const int64_t i = r0 + lane / TPV;
    T sum = 0;
    if (i < n) {
      const int s = rp[i], e = rp[i + 1];
      for (int k = s + sub; k < e; k += 2 * TPV) {
        const bool in2 = k + TPV < e;
        const int32_t c0 = ld_stream(ci + k);
        const int32_t c1 = in2 ? ld_stream(ci + k + TPV) : 0;
        const T w0 = ld_stream(v + k);
        const T w1 = in2 ? ld_stream(v + k + TPV) : T(0);
        sum = fma(w0, ld_x<COH>(x + c0), sum);
        if (in2) sum = fma(w1, ld_x<COH>(x + c1), sum);
      }
    }
#pragma unroll
    for (int o = TPV / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (sub == 0 && i < n) {
      store_row<T, GEN>(y, i, sum, alpha, beta);
      if (DOT) acc = fma(sum, COH ? ld_cg(dotv + i) : dotv[i], acc);
    }
  }
  return acc;
}

// ------------------------------------------------------------------ ELL
// Thread per row pair (i and i + stride); chunks of 4 slots give 16 independent
// coalesced loads before the gathers; padding (col -1) only follows a row's
// entries, so once both rows show padding the pair is done.
template <typename T, bool GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T ell_rows(int64_t n, int64_t K, int64_t ld,
                                      const int32_t* __restrict__ ec, const T* __restrict__ ev,
                                      const T* __restrict__ x, T* __restrict__ y, T alpha, T beta,
                                      const T* __restrict__ dotv, int64_t tid, int64_t stride) {
  T acc = 0;
  for (int64_t i0 = tid; i0 < n; i0 += 2 * stride) {
    const int64_t i1 = i0 + stride;
    const bool has1 = i1 < n;
    T s0 = 0, s1 = 0;
    for (int64_t k0 = 0; k0 < K; k0 += 4) {
      int32_t c0[4], c1[4];
      T w0[4], w1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = k0 + u < K;
        c0[u] = in ? ld_stream(ec + (k0 + u) * ld + i0) : -1;
        w0[u] = in ? ld_stream(ev + (k0 + u) * ld + i0) : T(0);
        c1[u] = (in && has1) ? ld_stream(ec + (k0 + u) * ld + i1) : -1;
        w1[u] = (in && has1) ? ld_stream(ev + (k0 + u) * ld + i1) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (c0[u] >= 0) s0 = fma(w0[u], ld_x<COH>(x + c0[u]), s0);
        if (c1[u] >= 0) s1 = fma(w1[u], ld_x<COH>(x + c1[u]), s1);
      }
      if (c0[3] < 0 && c1[3] < 0) break;
    }
    store_row<T, GEN>(y, i0, s0, alpha, beta);
    if (DOT) acc = fma(s0, COH ? ld_cg(dotv + i0) : dotv[i0], acc);
    if (has1) {
      store_row<T, GEN>(y, i1, s1, alpha, beta);
      if (DOT) acc = fma(s1, COH ? ld_cg(dotv + i1) : dotv[i1], acc);
    }
  }
  return acc;
}

// ------------------------------------------------------------------ SELL-C-sigma (C = 32)
// One warp per chunk, lane r on slot r: every load of the chunk is one
// contiguous 128-byte (col) and 256-byte (FP64 val) transaction.
template <typename T, bool GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T sell_chunks(int64_t n, int64_t nchunks,
                                         const int32_t* __restrict__ perm,
                                         const int32_t* __restrict__ clen,
                                         const int64_t* __restrict__ cptr,
                                         const int32_t* __restrict__ sc,
                                         const T* __restrict__ sv, const T* __restrict__ x,
                                         T* __restrict__ y, T alpha, T beta,
                                         const T* __restrict__ dotv, int64_t warp,
                                         int64_t nwarps) {
  const int lane = threadIdx.x & 31;
  T acc = 0;
  for (int64_t c = warp; c < nchunks; c += nwarps) {
    const int64_t base = cptr[c] + lane;
    const int w = clen[c];
    T sum = 0;
    for (int k0 = 0; k0 < w; k0 += 4) {
      int32_t cc[4];
      T vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = k0 + u < w;
        cc[u] = in ? ld_stream(sc + base + (int64_t)(k0 + u) * 32) : -1;
        vv[u] = in ? ld_stream(sv + base + (int64_t)(k0 + u) * 32) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (cc[u] >= 0) sum = fma(vv[u], ld_x<COH>(x + cc[u]), sum);
    }
    const int64_t s = c * 32 + lane;
    if (s < n) {
      const int64_t row = perm ? perm[s] : s;
      store_row<T, GEN>(y, row, sum, alpha, beta);
      if (DOT) acc = fma(sum, COH ? ld_cg(dotv + row) : dotv[row], acc);
    }
  }
  return acc;
}

// ------------------------------------------------------------------ DIA
// Thread per row pair (i and i + stride, so twice the loads in flight); so[]
// holds the offsets (in shared memory); values and x are read contiguously
// across the warp (no index arrays, no gather).  An FMA runs only for a real
// diagonal (a warp-uniform test), since FP64 FMAs are as scarce as bytes here.
template <typename T, bool GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T dia_rows(int64_t n, int64_t ncols, int ndiag, const int32_t* so,
                                      const T* __restrict__ dv, const T* __restrict__ x,
                                      T* __restrict__ y, T alpha, T beta,
                                      const T* __restrict__ dotv, int64_t tid, int64_t stride) {
  T acc = 0;
  for (int64_t i0 = tid; i0 < n; i0 += 2 * stride) {
    const int64_t i1 = i0 + stride;
    const bool has1 = i1 < n;
    T s0 = 0, s1 = 0;
    for (int d0 = 0; d0 < ndiag; d0 += 4) {
      T w0[4], x0[4], w1[4], x1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool real = d0 + u < ndiag;
        const int64_t off = real ? so[d0 + u] : 0;
        const int64_t c0 = i0 + off, c1 = i1 + off;
        const bool in0 = real && c0 >= 0 && c0 < ncols;
        const bool in1 = real && has1 && c1 >= 0 && c1 < ncols;
        const int64_t base = (int64_t)(d0 + u) * n;
        w0[u] = in0 ? ld_stream(dv + base + i0) : T(0);
        x0[u] = in0 ? ld_x<COH>(x + c0) : T(0);
        w1[u] = in1 ? ld_stream(dv + base + i1) : T(0);
        x1[u] = in1 ? ld_x<COH>(x + c1) : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (d0 + u < ndiag) {
          s0 = fma(w0[u], x0[u], s0);
          s1 = fma(w1[u], x1[u], s1);
        }
      }
    }
    store_row<T, GEN>(y, i0, s0, alpha, beta);
    if (DOT) acc = fma(s0, COH ? ld_cg(dotv + i0) : dotv[i0], acc);
    if (has1) {
      store_row<T, GEN>(y, i1, s1, alpha, beta);
      if (DOT) acc = fma(s1, COH ? ld_cg(dotv + i1) : dotv[i1], acc);
    }
  }
  return acc;
}

}  // namespace cp
