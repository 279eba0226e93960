// Shared declarations of the persistent CG kernel (cg_persist.cu) and its host
// driver (krylov.cu).
#pragma once

#include "internal.cuh"

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
};

enum {
  kPersistCsrScalar = 0,
  kPersistCsrVector = 1,
  kPersistEll = 2,
  kPersistSell = 3,
  kPersistDia = 4
};

template <typename T>
struct PersistArgs {
  int64_t n = 0;
  T *x = nullptr, *r = nullptr, *p = nullptr, *ap = nullptr;
  double *pa = nullptr, *pb = nullptr;  // block partials, capacity >= grid
  CgState* st = nullptr;
  Mirror* mir = nullptr;
  const volatile int* yield = nullptr;  // host-mapped: return at the next iteration boundary
  int it0 = 0, itmax = 0;
  double tol2 = 0.0;
  long long barrier_timeout_ns = 2000000000ll;
  // CSR
  const int32_t *rp = nullptr, *ci = nullptr;
  const T* v = nullptr;
  // ELL (or HYB without a COO part)
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
};

template <typename T>
struct PersistVals;
template <>
struct PersistVals<double> {
  static const double* csr(const cp_mat* m) { return m->val; }
  static const double* ell(const EllPart& e) { return e.val; }
  static const double* sell(const SellPart& s) { return s.val; }
  static const double* dia(const DiaPart& d) { return d.val; }
};
template <>
struct PersistVals<float> {
  static const float* csr(const cp_mat* m) { return m->val32; }
  static const float* ell(const EllPart& e) { return e.val32; }
  static const float* sell(const SellPart& s) { return s.val32; }
  static const float* dia(const DiaPart& d) { return d.val32; }
};

template <typename T>
bool persist_supported(const cp_mat* m, const cp_config& c);
// share = 1: the whole device; 2: half of every SM, leaving room for the
// side stream's feature / prediction / conversion kernels while they run.
template <typename T>
void persist_launch(cp_ctx* ctx, cp_mat* m, const cp_config& c, PersistArgs<T> a,
                    cudaStream_t s, int share);

}  // namespace cp
