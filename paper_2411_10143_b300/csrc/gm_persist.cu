// Persistent GMRES(m): the Arnoldi steps, the ends of cycles and the restarts
// of GMRES (Sec. I; Saad, Iterative Methods for Sparse Linear Systems, Alg. 6.9
// with Givens rotations) in one cooperative launch, one block of 1024 threads
// per SM.  Grid-wide barriers take the place of kernel boundaries.
//
// Rows.  Every block owns the rows that the format's grid-stride SpMV mapping
// gives its threads (BlockRows).  All vector work of a block (dot products,
// Gram-Schmidt subtraction, the update of x) runs over those same rows, so what
// a block's SpMV wrote is read back by the block after a __syncthreads: the
// first Gram-Schmidt pass needs no grid barrier after the SpMV.  (SELL with a
// row permutation is the exception and takes one; so do HYB with a COO part and
// COO, whose COO entries every block adds by atomics into a zeroed vector that
// each block then folds into its own rows.)
//
// Step j of a cycle, w = column j + 1 of V, orthogonalised by modified
// Gram-Schmidt in groups of g columns (g = 4 in FP64, 16 in FP32; see the
// grouped passes below) while the block's rows of w fit in shared memory:
//   1. w = A v_j; the block keeps its rows of w in shared memory and forms the
//      partials of (v_c, w) for the first group
//   2. per group: a grid reduction (every block sums the partials in the same
//      order, so every block gets the same bits), the group's coefficients by a
//      forward substitution with its inner products, then one pass that
//      subtracts the group and forms the next group's partials (after the last
//      group: ||w||^2 and the new column's inner products within its group)
//   3. thread 0 of every block forms the next Givens rotation and the residual
//      estimate |g_{j+1}| (a thread outside the passes has applied the earlier
//      rotations to the new Hessenberg column meanwhile); every block holds the
//      cycle's small matrices in shared memory and takes the same decisions
//      without further synchronisation.
// Systems whose rows of w do not fit (or gmres_orth = 1) take classical
// Gram-Schmidt instead:
//   1. w = A v_j; block partials of (v_c, w) for c <= j and of (w, w)
//   -- grid barrier
//   2. w -= sum_c h_c v_c; partials of ||w||^2, or (FP32) at once the block
//      partials of the second pass (v_c, w)
//   -- grid barrier
//   3. FP64: the second pass only when the first removed most of w,
//      ||w'||^2 < ||w||^2 / 2 (Daniel, Gragg, Kaufman and Stewart, 1976):
//      dots, barrier, subtraction, partials of ||w''||^2, barrier.  FP32 runs
//      the subtraction of its second pass here, then a barrier.
//   4. the Givens rotation as above.
// Columns are never normalised in place: column c of V holds v_c / s_c with
// the scale s_c kept in shared memory (1 / ||w|| of the step that made it), and
// the scales are folded into the SpMV's alpha, the dot products, the
// subtraction coefficients and the update of x.  That saves a pass over w per
// step.
//
// End of a cycle: y = R^-1 g by thread 0 of every block, x += V y over the
// block's rows, and unless the solve returns here, the restart r = b - A x
// (barrier, SpMV, barrier) with the true-residual convergence test.
//
// Returning to the host.  Block 0 reads the host-mapped yield flag each step
// and publishes it through the state; the kernel returns at the next step
// boundary (exit kind 1: columns normalised, the state readable by the
// per-step kernels, which carry on) or at the end of a cycle (kind 2: x
// updated).  It also returns at a cycle end when the iteration budget is spent
// or, without true_check, when the estimate reached tol.  Barrier waits are
// bounded (CP_ERR_TIMEOUT).
#include <cstdio>

#include "common.cuh"
#include "internal.cuh"
#include "gm_state.cuh"
#include "persist.cuh"
#include "spmv_rows.cuh"

namespace cp {

static_assert(kPersistBlock == 1024, "BlockRows assumes 1024-thread blocks");

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// The rows of block b: segments of L = 2^lshift consecutive rows starting at
// k S + b L (k = 0, 1, ...), S = grid L, cut at n.  Row f of the block (f <
// count) is row(f); rows increase with f.
struct BlockRows {
  int64_t base, S, count;
  int lshift;
  __device__ BlockRows(int64_t n, int lshift_, int64_t S_) : S(S_), lshift(lshift_) {
    base = (int64_t)blockIdx.x << lshift;
    const int64_t L = 1ll << lshift;
    if (base >= n) {
      count = 0;
    } else {
      const int64_t K = (n - base + S - 1) / S;  // segments that start below n
      const int64_t last = n - ((K - 1) * S + base);
      count = (K - 1) * L + (last < L ? last : L);
    }
  }
  __device__ __forceinline__ int64_t row(int64_t f) const {
    return (f >> lshift) * S + base + (f & ((1ll << lshift) - 1));
  }
};

// HYB with a COO part, and COO: the product's COO entries went to wc through
// atomics from every block; after a grid barrier each block adds its own rows
// into y (scaled like the rest of the product) and leaves wc zero again.
template <typename T>
__device__ __forceinline__ void fold_tail(const BlockRows& br, T* y, T* wc, T alpha) {
  for (int64_t f = threadIdx.x; f < br.count; f += blockDim.x) {
    const int64_t i = br.row(f);
    y[i] = fma(alpha, ld_cg(wc + i), ld_cg(y + i));
    wc[i] = T(0);
  }
  __syncthreads();
}

// Sums G values (G = 2, 4, 8 or 16) over the warp: at each of the first log2(G)
// exchanges a lane keeps half of its values and adds its partner's copies of
// them, then plain butterfly levels follow.  Lane l returns the warp total of
// value q = l / (32 / G).
template <int G, typename A>
__device__ __forceinline__ A warp_sum_group(A (&v)[G]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int n = G, sp = 16; n > 1; n >>= 1, sp >>= 1) {
    const bool hi = lane & sp;
#pragma unroll
    for (int u = 0; u < n / 2; ++u) {
      const A keep = hi ? v[u + n / 2] : v[u];
      const A send = hi ? v[u] : v[u + n / 2];
      v[u] = keep + __shfl_xor_sync(full, send, sp);
    }
  }
  A k = v[0];
#pragma unroll
  for (int sp = 16 / G; sp >= 1; sp >>= 1) k += __shfl_xor_sync(full, k, sp);
  return k;
}

// One warp's (group, chunk) units of block_dots: columns [c0, c0 + R) against
// w over the block's 32-row chunks [ch0, ch1); the four sums go to
// wp[(c0 + q) * 32 + warp].
template <typename T, int R>
__device__ __forceinline__ void dot_units(const BlockRows& br, const T* V, int64_t ldv, int c0,
                                          const T* w, int64_t ch0, int64_t ch1, double* wp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* vc = V + (int64_t)c0 * ldv;
  T acc[R];
#pragma unroll
  for (int q = 0; q < R; ++q) acc[q] = T(0);
  for (int64_t ch = ch0; ch < ch1; ++ch) {
    const int64_t f = ch * 32 + lane;
    if (f < br.count) {
      const int64_t i = br.row(f);
      const T wi = ld_cg(w + i);
      T v[R];
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = ld_cg(vc + q * ldv + i);
#pragma unroll
      for (int q = 0; q < R; ++q) acc[q] = fma(v[q], wi, acc[q]);
    }
  }
  double d[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int q = 0; q < R; ++q) d[q] = (double)acc[q];
  const double s = warp_sum_group<4, double>(d);
  const int q = (lane >> 3) & 3;
  if ((lane & 7) == 0 && q < R) wp[(c0 + q) * 32 + warp] = s;
}

// Block partials of (V_c, w), c < items, w = column wc of V (wc < items gives
// (w, w) as item wc): part[c * grid + block].  Items go four at a time
// (groups); the groups' 32-row chunks are dealt to the warps in equal
// contiguous runs, so a warp covers one or two groups.  The block total of an
// item is the fixed-order sum of its 32 warp slots (zero where a warp had no
// unit of that item).  wp: items * 32 doubles of shared memory.  Starts with a
// __syncthreads, which also orders the block's earlier writes of w.
template <typename T>
__device__ void block_dots(const BlockRows& br, const T* V, int64_t ldv, int items, int wc,
                           double* __restrict__ part, double* wp) {
  const int warp = threadIdx.x >> 5;
  __syncthreads();  // wp may still be read; the block's writes of w precede the reads
  for (int k = threadIdx.x; k < items * 32; k += blockDim.x) wp[k] = 0.0;
  __syncthreads();
  const int nG = (items + 3) >> 2;
  const int64_t nch = (br.count + 31) >> 5;
  const int64_t units = nG * nch;
  int64_t u = units * warp / 32;
  const int64_t u1 = units * (warp + 1) / 32;
  const T* w = V + (int64_t)wc * ldv;
  while (u < u1) {
    const int g = (int)(u / nch);
    const int64_t ch0 = u - g * nch;
    const int64_t take = (u1 - u) < (nch - ch0) ? (u1 - u) : (nch - ch0);
    const int c0 = 4 * g;
    const int R = items - c0 < 4 ? items - c0 : 4;
    switch (R) {
      case 1: dot_units<T, 1>(br, V, ldv, c0, w, ch0, ch0 + take, wp); break;
      case 2: dot_units<T, 2>(br, V, ldv, c0, w, ch0, ch0 + take, wp); break;
      case 3: dot_units<T, 3>(br, V, ldv, c0, w, ch0, ch0 + take, wp); break;
      default: dot_units<T, 4>(br, V, ldv, c0, w, ch0, ch0 + take, wp); break;
    }
    u += take;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < items; c += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < 32; ++k) s += wp[c * 32 + k];
    part[(int64_t)c * gridDim.x + blockIdx.x] = s;
  }
}

// out[c] = the grid's partials of item c summed (one warp per item, fixed
// order: every block gets the same bits), c < items; ends with a __syncthreads.
__device__ __forceinline__ void sum_items(const double* part, int items, double* out) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < items; c += nw) {
    const double s = warp_partials_cg(part + (int64_t)c * gridDim.x, gridDim.x);
    if ((threadIdx.x & 31) == 0) out[c] = s;
  }
  __syncthreads();
}

// w -= sum_{c < nc} coef[c] V_c over the block's rows, w = column wc; returns
// the thread's share of ||w||^2 (after the subtraction).
template <typename T>
__device__ __forceinline__ T block_sub(const BlockRows& br, T* V, int64_t ldv, int nc, int wc,
                                       const T* coef) {
  T acc = 0;
  T* w = V + (int64_t)wc * ldv;
  for (int64_t f = threadIdx.x; f < br.count; f += blockDim.x) {
    const int64_t i = br.row(f);
    T wi = ld_cg(w + i);
    for_slots(nc, [&](int64_t c0, auto R) {
      constexpr int r = decltype(R)::value;
      T v[r];
#pragma unroll
      for (int u = 0; u < r; ++u) v[u] = ld_cg(V + (c0 + u) * ldv + i);
#pragma unroll
      for (int u = 0; u < r; ++u) wi = fma(-coef[c0 + u], v[u], wi);
      return false;
    });
    w[i] = wi;
    acc = fma(wi, wi, acc);
  }
  return acc;
}

// Modified Gram-Schmidt in groups of G columns.  For unit vectors v_c the
// product of the projections (I - v_{c+G-1} v_{c+G-1}^T) ... (I - v_c v_c^T)
// equals I - V T V^T with V = [v_c .. v_{c+G-1}] and T = (I + L)^{-1}, L the
// strictly lower part of V^T V (the compact WY form, exact for any unit
// vectors).  So h = T V^T w, a forward substitution with the group's inner
// products (v_q, v_c), gives the coefficients modified Gram-Schmidt computes one
// column at a time, and the group costs one grid reduction instead of G.  A
// pass over the block's rows subtracts one group and forms the dot products of
// the next (or, after the last group, ||w||^2 and the new column's inner
// products with the columns of its own group, the entries of L its group will
// need).  G = 4 in FP64 (a pass holds 2G values a row in registers, and FP64
// halves what fits) and 16 in FP32, where the rounds' synchronisation, not the
// passes, is the larger cost: against groups of 8, 45.6 against 46.7 us a step
// on convection-diffusion 96^3 with DIA, 49.2 against 49.8 with ELL, although
// the FP32 passes spill about twice as much.
constexpr int kMgsThreads = 512;  // threads of a block that run the passes: half the
                                  // FP64 partials to reduce of 1024, and still
                                  // enough loads in flight (512 measured fastest of
                                  // 256 / 512 / 1024 on 884,736 rows)

template <typename T>
struct MgsGroup {
  static constexpr int value = sizeof(T) == 4 ? 16 : 4;
};

// Calls f(IntC<r>) for the runtime r in [R, MAX] (group sizes: exact register
// counts, no padding lanes of FP64 work).
template <int R, int MAX, typename F>
__device__ __forceinline__ void dispatch_r(int r, F&& f) {
  if constexpr (R >= MAX) {
    f(IntC<MAX>{});
  } else {
    if (r == R) f(IntC<R>{});
    else dispatch_r<R + 1, MAX>(r, f);
  }
}

template <typename T, int G, int RS, int RD, bool FIRST, bool LAST>
__device__ __forceinline__ void mgs_pass(const BlockRows& br, const T* V, int64_t ldv, int cs0,
                                         int cd0, const T* kc, T* ws, T* wg, T (&out)[G]) {
  T acc[G];
#pragma unroll
  for (int u = 0; u < G; ++u) acc[u] = T(0);
  T k[RS > 0 ? RS : 1];
#pragma unroll
  for (int u = 0; u < RS; ++u) k[u] = kc[u];
  for (int64_t f = threadIdx.x; f < br.count; f += kMgsThreads) {
    const int64_t i = br.row(f);
    T wv = FIRST ? ld_cg(wg + i) : ws[f];
    T a[RS > 0 ? RS : 1], d[RD > 0 ? RD : 1];
#pragma unroll
    for (int u = 0; u < RS; ++u) a[u] = ld_cg(V + (int64_t)(cs0 + u) * ldv + i);
#pragma unroll
    for (int u = 0; u < RD; ++u) d[u] = ld_cg(V + (int64_t)(cd0 + u) * ldv + i);
#pragma unroll
    for (int u = 0; u < RS; ++u) wv = fma(-k[u], a[u], wv);
    if (LAST) {
      wg[i] = wv;  // the next step's SpMV gathers it
      acc[0] = fma(wv, wv, acc[0]);
      if (RS < G) {
#pragma unroll
        for (int u = 0; u < RS; ++u) acc[1 + u] = fma(a[u], wv, acc[1 + u]);
      }
    } else {
      ws[f] = wv;
#pragma unroll
      for (int u = 0; u < RD; ++u) acc[u] = fma(d[u], wv, acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < G; ++u) out[u] = acc[u];
}

// The three kinds of pass: the first (w from global memory, dots of group 0),
// the middle ones (subtract a full group, dots of the next), the last
// (subtract the last group, ||w||^2 and the new column's group inner products).
template <typename T, int G>
__device__ __forceinline__ void mgs_first(int rd, const BlockRows& br, const T* V, int64_t ldv,
                                          T* ws, T* wg, T (&out)[G]) {
  dispatch_r<1, G>(rd, [&](auto R) {
    mgs_pass<T, G, 0, decltype(R)::value, true, false>(br, V, ldv, 0, 0, nullptr, ws, wg, out);
  });
}
template <typename T, int G>
__device__ __forceinline__ void mgs_mid(int rd, const BlockRows& br, const T* V, int64_t ldv,
                                        int cs0, const T* kc, T* ws, T* wg, T (&out)[G]) {
  dispatch_r<1, G>(rd, [&](auto R) {
    mgs_pass<T, G, G, decltype(R)::value, false, false>(br, V, ldv, cs0, cs0 + G, kc, ws, wg,
                                                        out);
  });
}
template <typename T, int G>
__device__ __forceinline__ void mgs_last(int rs, const BlockRows& br, const T* V, int64_t ldv,
                                         int cs0, const T* kc, T* ws, T* wg, T (&out)[G]) {
  dispatch_r<1, G>(rs, [&](auto R) {
    mgs_pass<T, G, decltype(R)::value, 0, false, true>(br, V, ldv, cs0, 0, kc, ws, wg, out);
  });
}

// min(max(v, 0), G): columns of a group that exist
template <int G>
__device__ __forceinline__ int clamp_group(int v) { return v < 0 ? 0 : (v > G ? G : v); }

// Block sums of G values held by the first kMgsThreads threads: each warp folds
// its G with warp_sum_group, then warp 0 adds the 16 warps' results of each value
// (32 / G lanes per value, a fixed tree) and writes the block's partials
// part[q * grid + block].  wp: G * 16 doubles.
template <typename T, int G>
__device__ __forceinline__ void mgs_block_partials(T (&v)[G], double* wp, double* part) {
  constexpr int nw = kMgsThreads / 32, LP = 32 / G;
  static_assert(nw == 16 && nw % LP == 0, "the tree below assumes 16 pass warps");
  if (threadIdx.x < kMgsThreads) {
    const double s = (double)warp_sum_group<G, T>(v);
    const int lane = threadIdx.x & 31;
    if ((lane & (LP - 1)) == 0) wp[(lane / LP) * nw + (threadIdx.x >> 5)] = s;
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // lane l: value l / LP; warp sums l % LP, l % LP + LP, ...
    const int q = threadIdx.x / LP, m = threadIdx.x & (LP - 1);
    double t = wp[q * nw + m];
#pragma unroll
    for (int k = m + LP; k < nw; k += LP) t += wp[q * nw + k];
#pragma unroll
    for (int sp = LP / 2; sp >= 1; sp >>= 1) t += __shfl_xor_sync(0xffffffffu, t, sp);
    if (m == 0) part[(int64_t)q * gridDim.x + blockIdx.x] = t;
  }
}

// Layout of the kernel's dynamic shared memory for restart length M, in
// doubles: the one description both the kernel's carving and the host's size use.
struct GmSmem {
  int64_t H, cs, sn, g, y, sc, h, h2, coef, wp, red, G, w, total;
  // wdoubles: doubles that hold a block's rows of w (modified Gram-Schmidt), or 0
  __host__ __device__ constexpr GmSmem(int M, int64_t wdoubles)
      : H(0),
        cs(H + (int64_t)(M + 1) * M),  // H: (M + 1) x M, H[i * M + j]
        sn(cs + M),
        g(sn + M),
        y(g + M + 1),
        sc(y + M),
        h(sc + M + 1),  // sc: M + 1 column scales
        h2(h + M + 2),
        coef(h2 + M + 2),
        wp(coef + M + 2),  // coef: M + 2 values of T (at most a double each)
        red(wp + 32 * (int64_t)(M + 2 > 4 ? M + 2 : 4)),  // wp: at least 128
        G(red + kPersistBlock + 4),  // G: (M + 1) x kMgsGroupMax group inner products
        w(G + kMgsGroupMax * (int64_t)(M + 1)),
        total(w + wdoubles) {}
};

template <typename T, int F, int TPV>
__global__ void __launch_bounds__(kPersistBlock, 1) k_gm_persist(GmPersistArgs<T> a) {
  GmState* st = a.st;
  // the solve ended, or the cycle ended in a step queued before this launch:
  // the host finishes the cycle
  if (ld_cg(&st->done) || ld_cg(&st->halt)) return;
  extern __shared__ double dsm[];
  const int M = a.mrest;
  const GmSmem L(M, a.wdoubles);
  double* H = dsm + L.H;    // rotated Hessenberg matrix of the cycle, H[i * M + j]
  double* cs = dsm + L.cs;  // Givens rotations
  double* sn = dsm + L.sn;
  double* g = dsm + L.g;    // rotated right-hand side
  double* yv = dsm + L.y;   // y = R^-1 g at the end of a cycle
  double* sc = dsm + L.sc;  // column c of V holds v_c / sc[c]
  double* h = dsm + L.h;    // first-pass coefficients, then (w, w)
  double* h2 = dsm + L.h2;  // second-pass coefficients
  T* coef = reinterpret_cast<T*>(dsm + L.coef);
  double* wp = dsm + L.wp;  // (M + 2) x 32 warp sums of block_dots
  double* red = dsm + L.red;
  constexpr int GS = MgsGroup<T>::value;  // columns per grid reduction
  double* G = dsm + L.G;    // (v_q, v_c) within groups of GS columns, G[q * GS + c % GS]
  T* ws = reinterpret_cast<T*>(dsm + L.w);  // the block's rows of w (modified Gram-Schmidt)
  __shared__ int32_t so[F == kPersistDia ? kDiaMax : 1];
  __shared__ double sh_w2;
  __shared__ double rsum[kMgsGroupMax];  // a grouped Gram-Schmidt round's sums
  __shared__ int sh_flag, sh_halt, sh_stop, sh_bad, sh_conv, sh_fin, sh_mcyc;

  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  const int64_t ldv = a.ldv;
  T* V = a.V;
  if constexpr (F == kPersistDia)
    for (int d = threadIdx.x; d < a.ndiag; d += blockDim.x) so[d] = a.offs[d];
  // the cycle so far (state of the per-step kernels: columns normalised)
  int j = ld_cg(&st->jdone);
  int iters = ld_cg(&st->iters);
  const int iters0 = iters;
  for (int k = threadIdx.x; k < (M + 1) * M; k += blockDim.x) {
    const int i = k / M, c = k - i * M;
    H[k] = ld_cg(&st->H[i * kMaxRestart + c]);
  }
  for (int k = threadIdx.x; k <= M; k += blockDim.x) {
    if (k < M) {
      cs[k] = ld_cg(&st->cs[k]);
      sn[k] = ld_cg(&st->sn[k]);
    }
    g[k] = ld_cg(&st->g[k]);
    sc[k] = 1.0;
  }
  for (int k = threadIdx.x; k < GS * (M + 1); k += blockDim.x)
    G[k] = ld_cg(&st->G[(k / GS) * kMgsGroupMax + k % GS]);
  if (lead) {
    st->mcyc = a.mcyc;
    a.mir->mcyc = a.mcyc;
  }
  int mcyc = a.mcyc;
  const double bb = ld_cg(&st->bb);
  __syncthreads();

  constexpr int lshift = F == kPersistCsrVector ? 10 - ilog2(TPV) : 10;
  const BlockRows br(a.n, lshift, (int64_t)gridDim.x << lshift);
  const bool fused = !(F == kPersistSell && a.perm != nullptr);
  unsigned bar_target = 0;
  auto barrier = [&]() {
    bar_target += gridDim.x;
    return grid_barrier(&st->bar_count, &st->bar_err, bar_target, a.barrier_timeout_ns);
  };
  unsigned long long tmark = lead ? global_ns() : 0;
  auto lap = [&](int k) {  // block 0's phase timer
    if (lead) {
      const unsigned long long now = global_ns();
      st->t_ns[k] += now - tmark;
      tmark = now;
    }
  };
  int exit_kind = 0;
  unsigned rounds = 0;  // grid reductions of the modified Gram-Schmidt loop so far
  for (;;) {
    T* w = V + (int64_t)(j + 1) * ldv;
    int second = 0;
    // the host's request (host-mapped, a bus round trip), read before the
    // SpMV so that the reduction that publishes it does not wait for it
    int yield = 0;
    if (lead) yield = *a.yield;
    if (a.mgs) {
      // ---- 1-3 (modified Gram-Schmidt in groups of GS): w = A v_j; per group
      // B_k = [GS k, GS k + R_k) one grid reduction of (v_c, w), then h_B = T_k (V_B^T w)
      // and w -= V_B h_B in the pass that forms the next group's dot products.
      // The block's rows of w stay in shared memory.
      persist_spmv<T, F, TPV, true, false>(a, so, V + (int64_t)j * ldv, w, (T)sc[j], T(0),
                                           nullptr);
      if constexpr (F == kPersistHyb) {
        coo_tail_atomic<T, false>(a, V + (int64_t)j * ldv, a.wc);
        if (!barrier()) break;
        fold_tail(br, w, a.wc, (T)sc[j]);
      } else if (!fused) {
        if (!barrier()) break;
      } else {
        __syncthreads();  // the block reads back the rows its threads wrote
      }
      const int nb = (j + GS) / GS;  // groups of the columns 0 .. j
      int rot = 0;                   // rotations applied to column j (helper thread)
      T part[GS];
#pragma unroll
      for (int u = 0; u < GS; ++u) part[u] = T(0);
      if (threadIdx.x < kMgsThreads)
        mgs_first<T, GS>(clamp_group<GS>(j + 1), br, V, ldv, ws, w, part);
      lap(0);
      bool ok = true;
      for (int k = 0;; ++k) {
        // partials alternate between two buffers over consecutive rounds, so a
        // round's writes never meet a slower block's reads of the round before
        double* pr = a.part + (int64_t)(rounds++ & 1) * GS * gridDim.x;
        if (k > 0) lap(2);  // passes
        mgs_block_partials<T, GS>(part, wp, pr);
        if (!barrier()) {
          ok = false;
          break;
        }
        if (k == 0 && lead) st->stop = yield || (a.chunk > 0 && iters + 1 - iters0 >= a.chunk);
        if (threadIdx.x < 32 * GS) {  // one warp per value
          const double t = warp_partials_cg(pr + (int64_t)(threadIdx.x >> 5) * gridDim.x,
                                            gridDim.x);
          if ((threadIdx.x & 31) == 0) rsum[threadIdx.x >> 5] = t;
        }
        __syncthreads();
        if (k == nb) break;  // rsum[0] = ||w||^2, rsum[1 ..] its group's raw inner products
        const int c0 = GS * k, R = j + 1 - c0 < GS ? j + 1 - c0 : GS;
        if (threadIdx.x < 32) {  // h_B = T_k r: forward substitution, lane i on h_{c0+i}
          const int i = threadIdx.x;
          double r = i < R ? rsum[i] * sc[c0 + i] : 0.0;
          for (int l = 0; l + 1 < R; ++l) {
            const double hl = __shfl_sync(0xffffffffu, r, l);
            if (i > l && i < R) r = fma(-G[(c0 + i) * GS + l], hl, r);
          }
          if (i < R) {
            h[c0 + i] = r;
            coef[i] = (T)(r * sc[c0 + i]);
          }
        }
        __syncthreads();
        lap(3);  // reductions, barriers, substitutions
        if (threadIdx.x == kMgsThreads) {
          // a thread outside the passes puts the group's coefficients into column j
          // of the Hessenberg matrix and applies the earlier Givens rotations as far
          // as the known entries allow, while the passes run
          for (int i = 0; i < R; ++i) H[(c0 + i) * M + j] = h[c0 + i];
          const int upto = c0 + R - 1 < j ? c0 + R - 1 : j;
          for (; rot < upto; ++rot) {
            const double p = H[rot * M + j], q = H[(rot + 1) * M + j];
            H[rot * M + j] = cs[rot] * p + sn[rot] * q;
            H[(rot + 1) * M + j] = -sn[rot] * p + cs[rot] * q;
          }
        }
        if (threadIdx.x < kMgsThreads) {
          if (k + 1 < nb) {
            mgs_mid<T, GS>(clamp_group<GS>(j + 1 - (c0 + GS)), br, V, ldv, c0, coef, ws, w,
                           part);
          } else {
            mgs_last<T, GS>(R, br, V, ldv, c0, coef, ws, w, part);
          }
        }
      }
      if (!ok) break;
      lap(3);
      if (threadIdx.x == 0) {  // the new column's inner products within its group
        sh_w2 = rsum[0];
        const int q = j + 1, r = q % GS;
        const double sq = rsum[0] > 0.0 ? 1.0 / sqrt(rsum[0]) : 0.0;
        for (int l = 0; l < GS; ++l) {
          const double gv = l < r ? rsum[1 + l] * sc[q - r + l] * sq : 0.0;
          G[q * GS + l] = gv;
          if (lead) st->G[q * kMgsGroupMax + l] = gv;
        }
      }
      lap(2);
    } else {
      // ---- 1. w = A v_j, first-pass dots
      persist_spmv<T, F, TPV, true, false>(a, so, V + (int64_t)j * ldv, w, (T)sc[j], T(0),
                                           nullptr);
      if constexpr (F == kPersistHyb) {
        coo_tail_atomic<T, false>(a, V + (int64_t)j * ldv, a.wc);
        if (!barrier()) break;
        fold_tail(br, w, a.wc, (T)sc[j]);
      }
      if (!fused && !barrier()) break;
      block_dots<T>(br, V, ldv, j + 2, j + 1, a.part, wp);
      lap(0);
      if (!barrier()) break;
      lap(1);
      // ---- 2. first subtraction
      // the host's request (or the end of the launch's chunk of steps), published
      // to every block by the next barrier
      if (lead) st->stop = yield || (a.chunk > 0 && iters + 1 - iters0 >= a.chunk);
      sum_items(a.part, j + 2, h);
      for (int c = threadIdx.x; c <= j; c += blockDim.x) {
        const double hc = h[c] * sc[c];  // (v_c, w)
        h[c] = hc;
        coef[c] = (T)(hc * sc[c]);
      }
      __syncthreads();
      const double ww = h[j + 1];
      {
        const T acc = block_sub<T>(br, V, ldv, j + 1, j + 1, coef);
        if (a.always_reorth) {
          block_dots<T>(br, V, ldv, j + 1, j + 1, a.part2, wp);
        } else {
          const double s = block_sum_lean((double)acc, red);
          if (threadIdx.x == 0) a.pn[blockIdx.x] = s;
        }
      }
      lap(2);
      if (!barrier()) break;
      lap(3);
      // ---- 3. second pass where needed
      second = a.always_reorth;
      if (!second) {
        if (threadIdx.x < 32) {
          const double w2 = warp_partials_cg(a.pn, gridDim.x);
          if (threadIdx.x == 0) {
            sh_w2 = w2;
            sh_flag = !(w2 >= 0.5 * ww);
          }
        }
        __syncthreads();
        second = sh_flag;
        if (second) {
          block_dots<T>(br, V, ldv, j + 1, j + 1, a.part2, wp);
          if (!barrier()) break;
        }
      }
      if (second) {
        sum_items(a.part2, j + 1, h2);
        for (int c = threadIdx.x; c <= j; c += blockDim.x) {
          const double hc = h2[c] * sc[c];
          h2[c] = hc;
          coef[c] = (T)(hc * sc[c]);
        }
        __syncthreads();
        const T acc = block_sub<T>(br, V, ldv, j + 1, j + 1, coef);
        const double s = block_sum_lean((double)acc, red);
        if (threadIdx.x == 0) a.pn[blockIdx.x] = s;
        if (!barrier()) break;
        if (threadIdx.x < 32) {
          const double w2 = warp_partials_cg(a.pn, gridDim.x);
          if (threadIdx.x == 0) sh_w2 = w2;
        }
      }
    }
    lap(4);
    // ---- 4. Givens rotation of column j (thread 0 of every block)
    if (threadIdx.x == 0) {
      const double hn2 = sh_w2;
      const double hn = sqrt(hn2);
      if (!a.mgs) {  // (the modified Gram-Schmidt branch has filled and rotated column j)
        for (int i = 0; i <= j; ++i) H[i * M + j] = h[i] + (second ? h2[i] : 0.0);
        for (int i = 0; i < j; ++i) {
          const double p = H[i * M + j], q = H[(i + 1) * M + j];
          H[i * M + j] = cs[i] * p + sn[i] * q;
          H[(i + 1) * M + j] = -sn[i] * p + cs[i] * q;
        }
      }
      const double p = H[j * M + j];
      const double den = sqrt(p * p + hn2);
      const double c = den == 0.0 ? 1.0 : p / den;
      const double s = den == 0.0 ? 0.0 : hn / den;
      cs[j] = c;
      sn[j] = s;
      H[j * M + j] = c * p + s * hn;
      g[j + 1] = -s * g[j];
      g[j] = c * g[j];
      const double est2 = g[j + 1] * g[j + 1];
      const bool bad = !isfinite(est2) || !isfinite(hn);
      const bool conv = est2 <= a.tol2 * bb;
      sc[j + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
      const bool halt = conv || hn == 0.0 || bad || j + 1 == mcyc;
      sh_bad = bad;
      sh_conv = conv;
      sh_halt = halt;
      sh_stop = *(volatile int*)&st->stop;
      if (lead) {
        for (int i = 0; i <= j; ++i) st->H[i * kMaxRestart + j] = H[i * M + j];
        st->cs[j] = c;
        st->sn[j] = s;
        st->g[j] = g[j];
        st->g[j + 1] = g[j + 1];
        st->inv = sc[j + 1];
        st->jdone = j + 1;
        st->iters = iters + 1;
        st->conv_est = conv ? 1 : 0;
        st->reorths += second ? 1 : 0;
        st->skip2 = second ? 0 : 1;
        if (bad) st->status = CP_ERR_BREAKDOWN;
        st->halt = halt ? 1 : 0;
        a.mir->res = fabs(g[j + 1]);
        a.mir->iters = iters + 1;
        a.mir->jdone = j + 1;
        a.mir->halt = halt ? 1 : 0;
        a.mir->conv_est = conv ? 1 : 0;
        if (bad) a.mir->status = CP_ERR_BREAKDOWN;
      }
    }
    __syncthreads();
    if (a.mgs) lap(1);
    ++iters;
    ++j;
    if (sh_bad) break;  // breakdown: the status is recorded
    if (!sh_halt) {
      if (sh_stop) {  // return inside the cycle: normalise the columns in place
        for (int64_t f = threadIdx.x; f < br.count; f += blockDim.x) {
          const int64_t i = br.row(f);
          for (int c = 0; c <= j; ++c) {
            const double s = sc[c];
            if (s != 1.0) V[(int64_t)c * ldv + i] = (T)(ld_cg(V + (int64_t)c * ldv + i) * s);
          }
        }
        exit_kind = 1;
        break;
      }
      continue;
    }
    // ---- end of the cycle: y = R^-1 g, x += V y
    if (threadIdx.x == 0) {
      for (int i = j - 1; i >= 0; --i) {
        double s = g[i];
        for (int k = i + 1; k < j; ++k) s -= H[i * M + k] * yv[k];
        yv[i] = s / H[i * M + i];
      }
      for (int c = 0; c < j; ++c) coef[c] = (T)(yv[c] * sc[c]);
      sh_fin = sh_stop || iters >= a.itmax || (sh_conv && !a.true_check);
    }
    __syncthreads();
    for (int64_t f = threadIdx.x; f < br.count; f += blockDim.x) {
      const int64_t i = br.row(f);
      T xi = ld_cg(a.x + i);
      for_slots(j, [&](int64_t c0, auto R) {
        constexpr int r = decltype(R)::value;
        T v[r];
#pragma unroll
        for (int u = 0; u < r; ++u) v[u] = ld_cg(V + (c0 + u) * ldv + i);
#pragma unroll
        for (int u = 0; u < r; ++u) xi = fma(coef[c0 + u], v[u], xi);
        return false;
      });
      a.x[i] = xi;
    }
    if (sh_fin) {
      exit_kind = 2;
      break;
    }
    if (!barrier()) break;
    // ---- restart: r = b - A x into column 0, the true-residual test
    persist_spmv<T, F, TPV, false, false>(a, so, a.x, V, T(1), T(0), nullptr);
    if constexpr (F == kPersistHyb) {
      coo_tail_atomic<T, false>(a, a.x, a.wc);
      if (!barrier()) break;
      fold_tail(br, V, a.wc, T(1));
    } else if (!fused) {
      if (!barrier()) break;
    } else {
      __syncthreads();
    }
    {
      T acc = 0;
      for (int64_t f = threadIdx.x; f < br.count; f += blockDim.x) {
        const int64_t i = br.row(f);
        const T r = ld_cg(a.b + i) - ld_cg(V + i);
        V[i] = r;
        acc = fma(r, r, acc);
      }
      const double s = block_sum_lean((double)acc, red);
      if (threadIdx.x == 0) a.pn[blockIdx.x] = s;
    }
    if (!barrier()) break;
    if (threadIdx.x < 32) {
      const double rr = warp_partials_cg(a.pn, gridDim.x);
      if (threadIdx.x == 0) {
        const double beta = sqrt(rr);
        const bool conv = bb == 0.0 || rr <= a.tol2 * bb;
        const bool bad = !isfinite(rr);
        const int m_next = a.itmax - iters < M ? a.itmax - iters : M;
        sh_fin = conv || bad;
        sh_mcyc = m_next;
        sc[0] = beta > 0.0 ? 1.0 / beta : 0.0;
        g[0] = beta;
        for (int k = 1; k <= M; ++k) g[k] = 0.0;
        for (int k = 0; k < GS * (M + 1); ++k) G[k] = 0.0;
        if (lead) {
          st->beta = beta;
          st->g[0] = beta;
          for (int k = 1; k <= kMaxRestart; ++k) st->g[k] = 0.0;
          for (int k = 0; k < kMgsGroupMax * (kMaxRestart + 1); ++k) st->G[k] = 0.0;
          st->inv = sc[0];
          st->jdone = 0;
          st->conv_est = 0;
          st->mcyc = m_next;
          if (bad) st->status = CP_ERR_BREAKDOWN;
          st->done = sh_fin;
          st->halt = sh_fin;
          a.mir->res = beta;
          a.mir->jdone = 0;
          a.mir->conv_est = 0;
          a.mir->mcyc = m_next;
          if (bad) a.mir->status = CP_ERR_BREAKDOWN;
          a.mir->halt = sh_fin;
          a.mir->done = sh_fin;
        }
      }
    }
    __syncthreads();
    lap(5);
    if (sh_fin) break;
    mcyc = sh_mcyc;
    j = 0;
  }
  if (lead) {
    if (*(volatile int*)&st->bar_err) {
      st->status = CP_ERR_TIMEOUT;
      st->done = 1;
      a.mir->status = CP_ERR_TIMEOUT;
      a.mir->done = 1;
    }
    a.mir->exit_kind = exit_kind;
  }
}

// ------------------------------------------------------------------ host
// The launch: one 1024-thread block per SM.  The kernel orthogonalises with
// modified Gram-Schmidt in groups of four when a block's rows of w fit in shared
// memory next to the cycle's small matrices (FP64: n up to about three million
// rows at m = 30, FP32 twice that): half the FMAs and passes of classical
// Gram-Schmidt applied twice, for one grid reduction per group.  Larger systems
// take classical Gram-Schmidt with the second pass (conditional in FP64, in
// every step in FP32).
template <typename T, int F, int TPV>
static void gm_launch_one(cp_ctx* ctx, GmPersistArgs<T>& a, cudaStream_t s) {
  auto kern = k_gm_persist<T, F, TPV>;
  const int grid = ctx->num_sms < kMaxPartials ? ctx->num_sms : kMaxPartials;
  constexpr int lshift = F == kPersistCsrVector ? 10 - ilog2(TPV) : 10;
  const int64_t L = 1ll << lshift, S = (int64_t)grid * L;
  const int64_t wrows = (a.n + S - 1) / S * L;  // most rows a block owns
  cudaFuncAttributes fa{};
  CP_CUDA(cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(kern)));
  int optin = 0;
  CP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  const size_t room = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  const bool want_mgs = a.mgs != 0;
  a.mgs = 0;
  a.wdoubles = 0;
  const int64_t wdoubles = (wrows * (int64_t)sizeof(T) + 7) / 8;  // w region, in doubles
  if (want_mgs && (size_t)GmSmem(a.mrest, wdoubles).total * sizeof(double) <= room) {
    a.mgs = 1;
    a.wdoubles = wdoubles;
  }
  const size_t smem = (size_t)GmSmem(a.mrest, a.wdoubles).total * sizeof(double);
  CP_REQUIRE(smem <= room, CP_ERR_UNSUPPORTED, "persistent GMRES: restart too long for shared memory");
  CP_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(kern),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersistBlock, smem));
  CP_REQUIRE(per_sm >= 1, CP_ERR_CUDA, "persistent GMRES kernel does not fit an SM");
  void* args[] = {&a};
  CP_CUDA(cudaMemsetAsync(&a.st->bar_count, 0, sizeof(unsigned), s));
  CP_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid),
                                      dim3(kPersistBlock), args, smem, s));
  ctx->launches.fetch_add(1, std::memory_order_relaxed);
  trace("persistent GMRES: %s, %d blocks, %zu bytes of shared memory",
        a.mgs ? "modified Gram-Schmidt" : "classical Gram-Schmidt", grid, smem);
}

template <typename T>
bool gm_persist_supported(const cp_mat* m, const cp_config& c, int mrest) {
  return persist_format_ok(m, c, true) && mrest >= 1 && mrest <= kMaxRestart;
}

template <typename T>
void gm_persist_launch(cp_ctx* ctx, cp_mat* m, const cp_config& c, GmPersistArgs<T> a,
                       cudaStream_t s) {
  persist_dispatch<T, true>(m, c, a, [&](auto f, auto tpv) {
    gm_launch_one<T, decltype(f)::value, decltype(tpv)::value>(ctx, a, s);
  });
}

template bool gm_persist_supported<double>(const cp_mat*, const cp_config&, int);
template bool gm_persist_supported<float>(const cp_mat*, const cp_config&, int);
template void gm_persist_launch<double>(cp_ctx*, cp_mat*, const cp_config&,
                                        GmPersistArgs<double>, cudaStream_t);
template void gm_persist_launch<float>(cp_ctx*, cp_mat*, const cp_config&, GmPersistArgs<float>,
                                       cudaStream_t);

}  // namespace cp
