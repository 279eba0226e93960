// GMRES(m) state and the persistent GMRES kernel's arguments (gm_persist.cu),
// shared with the per-step kernels and the host driver (krylov.cu).
#pragma once

#include "persist.cuh"

namespace cp {

constexpr int kMaxRestart = 64;  // largest GMRES restart length

// GMRES(m) state of one solve (Sec. I; Saad, Alg. 6.9): the rotated Hessenberg
// matrix, the Givens rotations and the rotated right-hand side g of the current
// cycle, written by the per-step kernels and by the persistent kernel's block 0.
// Stride of the Gram entries G below: the largest group of the persistent
// kernel's modified Gram-Schmidt.
constexpr int kMgsGroupMax = 16;

struct GmState {
  double h1[kMaxRestart + 1], h2[kMaxRestart + 1];
  double H[(kMaxRestart + 1) * kMaxRestart];  // rotated Hessenberg, H[i * kMaxRestart + j]
  double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
  // inner products (v_q, v_c) of column q with the columns c before it in its
  // aligned group of g columns (g = 4 in FP64, 16 in FP32), G[q * kMgsGroupMax + (c - g
  // floor(q / g))]: the persistent kernel's modified Gram-Schmidt applies a
  // group's projections in one pass with them.  Zero for columns made by the
  // per-step kernels (orthogonal to working precision by the second
  // Gram-Schmidt pass).
  double G[(kMaxRestart + 1) * kMgsGroupMax];
  double bb, beta, inv;  // ||b||^2, cycle start ||r||, 1 / current norm
  int done;              // converged (true residual of a cycle start)
  int halt;              // no further steps in this cycle
  int conv_est;          // the cycle's residual estimate reached tol
  int jdone;             // steps completed in this cycle
  int status;
  int iters;             // steps completed in total
  int skip2;             // this step's second Gram-Schmidt pass is not needed
  int reorths;           // steps that took the second pass
  int mcyc;              // length of the current cycle (min(m, iterations left at its start))
  int stop;              // persistent kernel: return at the next step boundary
  unsigned bar_count;    // persistent kernel: barrier arrivals (this launch)
  int bar_err;           // persistent kernel: a barrier wait gave up
  // block 0's time in the persistent kernel (ns).  Classical Gram-Schmidt: SpMV
  // + first dots, barrier, subtraction, barrier, second pass, end of cycle;
  // modified: SpMV + first dots, Givens, passes, reductions, -, end of cycle
  // (the host's trace prints them per step)
  unsigned long long t_ns[6];
};

template <typename T>
struct GmPersistArgs : PersistMat<T> {
  T* V = nullptr;  // basis, column c at V + c * ldv; column jdone holds the next vector
  int64_t ldv = 0;
  T* x = nullptr;
  const T* b = nullptr;
  T* wc = nullptr;  // HYB / COO: the COO entries' part of a product, zero between products
  double *part = nullptr, *part2 = nullptr;  // (m + 2) x grid block partials each
  double* pn = nullptr;                      // grid block partials
  GmState* st = nullptr;
  Mirror* mir = nullptr;
  const volatile int* yield = nullptr;  // host-mapped: return at the next step boundary
  int itmax = 0;         // iteration budget (total steps)
  int mrest = 0;         // restart length m
  int mcyc = 0;          // length of the cycle the launch enters
  int chunk = 0;         // > 0: return at the step boundary after this many steps
  int mgs = 0;           // host: modified Gram-Schmidt wanted; kernel: in use (w in shared memory)
  int64_t wdoubles = 0;  // with mgs: shared-memory doubles that hold a block's rows of w
  int true_check = 1;    // 0: a cycle whose estimate reached tol ends the solve (FP32 inner solves)
  int always_reorth = 0; // second Gram-Schmidt pass in every step (FP32)
  double tol2 = 0.0;
  long long barrier_timeout_ns = 2000000000ll;
};

template <typename T>
bool gm_persist_supported(const cp_mat* m, const cp_config& c, int mrest);
template <typename T>
void gm_persist_launch(cp_ctx* ctx, cp_mat* m, const cp_config& c, GmPersistArgs<T> a,
                       cudaStream_t s);

}  // namespace cp
