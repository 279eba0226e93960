// Row loops of the row-parallel SpMV formats (CSR-scalar, CSR-vector, ELL,
// SELL-C-sigma, DIA).  Each walks its rows grid-stride from the caller's
// thread (or warp) index, writes y = A x (or alpha A x + beta y) and returns the
// thread's share of sum_i (A x)_i * dotv_i when DOT is set; the two-barrier
// persistent CG kernel also runs its direction update in them (kRowCgRec).  The
// SpMV kernels of spmv.cu wrap them one launch each; the persistent kernels run
// them as the SpMV phase of every iteration with COH set, so the x and dot
// vectors (which those kernels rewrite every iteration) never come from the
// read-only path: x through L1 after the grid barrier's acquire (ld_x), the
// dot vector through L2.
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

// What a row loop does with a finished row sum s = (A x)_i (its GEN argument):
constexpr int kRowSolve = 0;  // y_i = s; DOT: the share of sum s dotv_i
constexpr int kRowGen = 1;    // y_i = alpha s + beta y_i; DOT: the share of sum s dotv_i
// The persistent CG kernel's fused direction step, x being r+ and y the
// previous A p: y_i = s + beta y_i (A p+ = A r+ + beta A p), pw_i = r+_i +
// beta pw_i (p+ = r+ + beta p); returns the share of (p+, A p+).  Every value
// goes through L2 (the kernel's other phases write them on other SMs).
constexpr int kRowCgRec = 2;

// The operands of a row's kRowCgRec epilogue (y_i, pw_i, x_i), loaded with the
// row's first loads, so that a trip of the row loop waits for one memory round
// trip rather than two (the sum's loads, then the epilogue's).  Empty in the
// other modes.
template <typename T, int GEN>
struct RowPre {
  T q, p, r;
  __device__ __forceinline__ void load(const T* y, const T* pw, const T* x, int64_t i) {
    if constexpr (GEN == kRowCgRec) {
      q = ld_cg(y + i);
      p = ld_cg(pw + i);
      r = ld_cg(x + i);
    }
  }
};

template <typename T, int GEN, bool DOT, bool COH>
__device__ __forceinline__ T finish_row(T* __restrict__ y, int64_t i, T s, T alpha, T beta,
                                        const T* __restrict__ dotv, T* __restrict__ pw,
                                        const RowPre<T, GEN>& pre, T acc) {
  if constexpr (GEN == kRowCgRec) {
    const T q = fma(beta, pre.q, s);
    const T p = fma(beta, pre.p, pre.r);
    y[i] = q;
    pw[i] = p;
    return fma(p, q, acc);
  } else {
    store_row<T, GEN != kRowSolve>(y, i, s, alpha, beta);
    if (DOT) acc = fma(s, COH ? ld_cg(dotv + i) : dotv[i], acc);
    return acc;
  }
}

// ------------------------------------------------------------------ CSR scalar
// One thread per row; entries in chunks of 4 so the 8 index / value loads are
// independent, then 4 gathers.
template <typename T, int GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T csr_scalar_rows(int64_t n, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci,
                                             const T* __restrict__ v, const T* __restrict__ x,
                                             T* __restrict__ y, T alpha, T beta,
                                             const T* __restrict__ dotv, int64_t tid,
                                             int64_t stride, T* __restrict__ pw = nullptr) {
  T acc = 0;
  for (int64_t i = tid; i < n; i += stride) {
    RowPre<T, GEN> pre;
    pre.load(y, pw, x, i);
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
    acc = finish_row<T, GEN, DOT, COH>(y, i, sum, alpha, beta, dotv, pw, pre, acc);
  }
  return acc;
}

// ------------------------------------------------------------------ CSR vector
// TPV lanes per row; the warp walks its rows in lock step so the shuffles of
// the row reduction always see the full warp.  warp / nwarps: global warp index
// and count.
template <typename T, int TPV, int GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T csr_vector_rows(int64_t n, const int32_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci,
                                             const T* __restrict__ v, const T* __restrict__ x,
                                             T* __restrict__ y, T alpha, T beta,
                                             const T* __restrict__ dotv, int64_t warp,
                                             int64_t nwarps, T* __restrict__ pw = nullptr) {
  constexpr int RPW = 32 / TPV;  // rows per warp step
  const int lane = threadIdx.x & 31;
  const int sub = lane % TPV;
  T acc = 0;
  for (int64_t r0 = warp * RPW; r0 < n; r0 += nwarps * RPW) {
    const int64_t i = r0 + lane / TPV;
    RowPre<T, GEN> pre;
    if (sub == 0 && i < n) pre.load(y, pw, x, i);
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
      acc = finish_row<T, GEN, DOT, COH>(y, i, sum, alpha, beta, dotv, pw, pre, acc);
    }
  }
  return acc;
}

// Compile-time slot count for the unrolled loops below.
template <int R>
struct Slots {
  static constexpr int value = R;
};

// Runs f(k0, Slots<4>) over the full chunks of 4 slots in [0, w), then once
// with the exact remainder (1 to 3 slots).  w is the same in every lane of the
// warp (ELL width, a SELL chunk's width, the DIA diagonal count), so the
// remainder branch is uniform and no padding slot issues a predicated-off FMA:
// where the FP64 pipe bounds the kernel, a slot with no work costs as much as
// one with work.  f returns true to stop early.
template <typename F>
__device__ __forceinline__ void for_slots(int64_t w, F&& f) {
  int64_t k0 = 0;
  for (; k0 + 4 <= w; k0 += 4)
    if (f(k0, Slots<4>{})) return;
  switch (w - k0) {
    case 3: f(k0, Slots<3>{}); break;
    case 2: f(k0, Slots<2>{}); break;
    case 1: f(k0, Slots<1>{}); break;
    default: break;
  }
}

// The same with chunks of 8 slots (remainder 1 to 7): twice the loads in flight
// per chunk, for loops whose values take one register each (FP32), where the
// row loop is bound by memory latency rather than by the FMA pipe.
template <typename F>
__device__ __forceinline__ void for_slots8(int64_t w, F&& f) {
  int64_t k0 = 0;
  for (; k0 + 8 <= w; k0 += 8)
    if (f(k0, Slots<8>{})) return;
  switch (w - k0) {
    case 7: f(k0, Slots<7>{}); break;
    case 6: f(k0, Slots<6>{}); break;
    case 5: f(k0, Slots<5>{}); break;
    case 4: f(k0, Slots<4>{}); break;
    case 3: f(k0, Slots<3>{}); break;
    case 2: f(k0, Slots<2>{}); break;
    case 1: f(k0, Slots<1>{}); break;
    default: break;
  }
}

// Chunks of 8 for FP32 values, 4 for FP64 (whose loops the FP64 pipe bounds,
// and whose registers are twice as scarce).
template <typename T, typename F>
__device__ __forceinline__ void for_slots_t(int64_t w, F&& f) {
  if constexpr (sizeof(T) == 4) for_slots8(w, f);
  else for_slots(w, f);
}

// ------------------------------------------------------------------ ELL
// Thread per row pair (i and i + stride); chunks of 4 slots give 16 independent
// coalesced loads before the gathers; padding (col -1) only follows a row's
// entries, so once both rows show padding the pair is done.
template <typename T, int GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T ell_rows(int64_t n, int64_t K, int64_t ld,
                                      const int32_t* __restrict__ ec, const T* __restrict__ ev,
                                      const T* __restrict__ x, T* __restrict__ y, T alpha, T beta,
                                      const T* __restrict__ dotv, int64_t tid, int64_t stride,
                                      T* __restrict__ pw = nullptr) {
  T acc = 0;
  for (int64_t i0 = tid; i0 < n; i0 += 2 * stride) {
    const int64_t i1 = i0 + stride;
    const bool has1 = i1 < n;
    RowPre<T, GEN> pre0, pre1;
    pre0.load(y, pw, x, i0);
    if (has1) pre1.load(y, pw, x, i1);
    T s0 = 0, s1 = 0;
    for_slots_t<T>(K, [&](int64_t k0, auto R) {
      constexpr int r = decltype(R)::value;
      int32_t c0[r], c1[r];
      T w0[r], w1[r];
#pragma unroll
      for (int u = 0; u < r; ++u) {
        c0[u] = ld_stream(ec + (k0 + u) * ld + i0);
        w0[u] = ld_stream(ev + (k0 + u) * ld + i0);
        c1[u] = has1 ? ld_stream(ec + (k0 + u) * ld + i1) : -1;
        w1[u] = has1 ? ld_stream(ev + (k0 + u) * ld + i1) : T(0);
      }
#pragma unroll
      for (int u = 0; u < r; ++u) {
        if (c0[u] >= 0) s0 = fma(w0[u], ld_x<COH>(x + c0[u]), s0);
        if (c1[u] >= 0) s1 = fma(w1[u], ld_x<COH>(x + c1[u]), s1);
      }
      return c0[r - 1] < 0 && c1[r - 1] < 0;
    });
    acc = finish_row<T, GEN, DOT, COH>(y, i0, s0, alpha, beta, dotv, pw, pre0, acc);
    if (has1) {
      acc = finish_row<T, GEN, DOT, COH>(y, i1, s1, alpha, beta, dotv, pw, pre1, acc);
    }
  }
  return acc;
}

// ------------------------------------------------------------------ SELL-C-sigma (C = 32)
// One warp per chunk, lane r on slot r: every load of the chunk is one
// contiguous 128-byte (col) and 256-byte (FP64 val) transaction.
template <typename T, int GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T sell_chunks(int64_t n, int64_t nchunks,
                                         const int32_t* __restrict__ perm,
                                         const int32_t* __restrict__ clen,
                                         const int64_t* __restrict__ cptr,
                                         const int32_t* __restrict__ sc,
                                         const T* __restrict__ sv, const T* __restrict__ x,
                                         T* __restrict__ y, T alpha, T beta,
                                         const T* __restrict__ dotv, int64_t warp,
                                         int64_t nwarps, T* __restrict__ pw = nullptr) {
  const int lane = threadIdx.x & 31;
  T acc = 0;
  for (int64_t c = warp; c < nchunks; c += nwarps) {
    const int64_t base = cptr[c] + lane;
    const int64_t s = c * 32 + lane;
    const int64_t row = s < n ? (perm ? perm[s] : s) : -1;
    RowPre<T, GEN> pre;
    if (row >= 0) pre.load(y, pw, x, row);
    T sum = 0;
    for_slots_t<T>(clen[c], [&](int64_t k0, auto R) {
      constexpr int r = decltype(R)::value;
      int32_t cc[r];
      T vv[r];
#pragma unroll
      for (int u = 0; u < r; ++u) {
        cc[u] = ld_stream(sc + base + (k0 + u) * 32);
        vv[u] = ld_stream(sv + base + (k0 + u) * 32);
      }
#pragma unroll
      for (int u = 0; u < r; ++u)
        if (cc[u] >= 0) sum = fma(vv[u], ld_x<COH>(x + cc[u]), sum);
      return false;
    });
    if (row >= 0) acc = finish_row<T, GEN, DOT, COH>(y, row, sum, alpha, beta, dotv, pw, pre, acc);
  }
  return acc;
}

// ------------------------------------------------------------------ DIA
// Persistent kernels gather x through L1 (ld_x), except in FP64: there the FP64
// pipe bounds the loop, and the reuse of the neighbouring diagonals' lines in
// L1 measured 0.4 % slower than L2 alone (3D Poisson 128^3, FP64 CG: 59.5
// against 59.2 us an iteration; FP32 inner CG 27.1 against 27.5 us).
template <typename T>
constexpr bool kDiaL2 = sizeof(T) == 8;

// Thread per row pair (i and i + stride, so twice the loads in flight); so[]
// holds the offsets (in shared memory); values and x are read contiguously
// across the warp (no index arrays, no gather).  Every diagonal slot is real
// (exact remainder chunk), since FP64 FMAs are as scarce as bytes here.
template <typename T, int GEN, bool DOT, bool COH = false>
__device__ __forceinline__ T dia_rows(int64_t n, int64_t ncols, int ndiag, const int32_t* so,
                                      const T* __restrict__ dv, const T* __restrict__ x,
                                      T* __restrict__ y, T alpha, T beta,
                                      const T* __restrict__ dotv, int64_t tid, int64_t stride,
                                      T* __restrict__ pw = nullptr) {
  T acc = 0;
  // rows i with every i + offset inside [0, ncols) (all but a band at each end
  // for a stencil) take a loop without per-slot bounds checks
  int32_t omin = 0, omax = 0;
  for (int d = 0; d < ndiag; ++d) {
    const int32_t o = so[d];
    omin = o < omin ? o : omin;
    omax = o > omax ? o : omax;
  }
  const int64_t lo = -(int64_t)omin, hi = ncols - (int64_t)omax;
  for (int64_t i0 = tid; i0 < n; i0 += 2 * stride) {
    const int64_t i1 = i0 + stride;
    const bool has1 = i1 < n;
    T s0 = 0, s1 = 0;
    if (has1 && i0 >= lo && i1 < hi) {
      for_slots_t<T>(ndiag, [&](int64_t d0, auto R) {
        constexpr int r = decltype(R)::value;
        T w0[r], x0[r], w1[r], x1[r];
#pragma unroll
        for (int u = 0; u < r; ++u) {
          const int64_t off = so[d0 + u];
          const int64_t base = (d0 + u) * n;
          w0[u] = ld_stream(dv + base + i0);
          x0[u] = ld_x<COH, kDiaL2<T>>(x + i0 + off);
          w1[u] = ld_stream(dv + base + i1);
          x1[u] = ld_x<COH, kDiaL2<T>>(x + i1 + off);
        }
#pragma unroll
        for (int u = 0; u < r; ++u) {
          s0 = fma(w0[u], x0[u], s0);
          s1 = fma(w1[u], x1[u], s1);
        }
        return false;
      });
    } else {
      for_slots_t<T>(ndiag, [&](int64_t d0, auto R) {
        constexpr int r = decltype(R)::value;
        T w0[r], x0[r], w1[r], x1[r];
#pragma unroll
        for (int u = 0; u < r; ++u) {
          const int64_t off = so[d0 + u];
          const int64_t c0 = i0 + off, c1 = i1 + off;
          const bool in0 = c0 >= 0 && c0 < ncols;
          const bool in1 = has1 && c1 >= 0 && c1 < ncols;
          const int64_t base = (d0 + u) * n;
          w0[u] = in0 ? ld_stream(dv + base + i0) : T(0);
          x0[u] = in0 ? ld_x<COH, kDiaL2<T>>(x + c0) : T(0);
          w1[u] = in1 ? ld_stream(dv + base + i1) : T(0);
          x1[u] = in1 ? ld_x<COH, kDiaL2<T>>(x + c1) : T(0);
        }
#pragma unroll
        for (int u = 0; u < r; ++u) {
          s0 = fma(w0[u], x0[u], s0);
          s1 = fma(w1[u], x1[u], s1);
        }
        return false;
      });
    }
    // the epilogue's operands are loaded after the sums here: loaded with the
    // trip's first loads, they made the FP32 loop spill (126 against 78 bytes)
    // and cost 29.6 against 27.2 us a CG iteration on 3D Poisson 128^3
    RowPre<T, GEN> pre0, pre1;
    pre0.load(y, pw, x, i0);
    acc = finish_row<T, GEN, DOT, COH>(y, i0, s0, alpha, beta, dotv, pw, pre0, acc);
    if (has1) {
      pre1.load(y, pw, x, i1);
      acc = finish_row<T, GEN, DOT, COH>(y, i1, s1, alpha, beta, dotv, pw, pre1, acc);
    }
  }
  return acc;
}

}  // namespace cp
