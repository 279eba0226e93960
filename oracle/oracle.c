/*
 * CPU oracle for the cascaded-prediction Krylov hot path (arXiv 2411.10143).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file: only the test suite, the graft smoke check and the
 * benchmark's CPU-baseline leg may use it.  It shares no code, header, table
 * or constant with the CUDA path.
 *
 * Everything here is plain, single-threaded, FP64 C written for readability
 * against the definitions it follows, not for speed:
 *   - SpMV: the CSR definition y_i = sum_k val[k] x[col[k]] (Sec. I, Eq. of
 *     SpMV as the kernel both Krylov methods spend most time in).
 *   - CG: Hestenes-Stiefel conjugate gradient (Sec. I names CG; algorithm as in
 *     Saad, "Iterative Methods for Sparse Linear Systems", Alg. 6.18).
 *   - GMRES(m): restarted GMRES with modified Gram-Schmidt Arnoldi and Givens
 *     rotations (Sec. I / Sec. IV-A; Saad Alg. 6.9 and Sec. 6.5.3).
 *   - the 15 sparse-matrix features of Table IV (Sec. III-B-1).
 *   - canonical CSR -> COO / ELL / SELL-C-sigma / HYB layouts and their inverses
 *     (the format space of Sec. III-B-2 and the slicing of Sec. V-A).
 *   - mixed-precision iterative refinement with FP32 inner solves (FP32 emulated
 *     with C float, IEEE round-to-nearest-even on every cast).
 *   - the predictor MLP: forward pass, softmax cross-entropy loss, analytic
 *     backward pass and one Adam step, in FP64 (Sec. III-B-3 trains a
 *     classifier per cascade stage; this build uses small MLPs).
 *
 * Parity status of each function is stated in its comment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int32_t i32;
typedef int64_t i64;

/* The pragmas below mark the row-parallel SpMV and the vector loops of CG for
 * the second, all-core build of this same file (gcc -fopenmp, used only as a
 * timing baseline).  The oracle itself is built without -fopenmp: the pragmas
 * are then ignored and every loop runs serially in the order written.        */
/* ------------------------------------------------------------------------- */
/* SpMV (definition).  Pinned: brute-force dense matvec, exact integer data.  */
/* ------------------------------------------------------------------------- */
void or_spmv(i64 n, const i32* rowptr, const i32* col, const double* val,
             const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) {
    double s = 0.0;
    for (i64 k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = s;
  }
}

/* FP32 SpMV (values, x and the sum all in float): the inner-solve operator of
 * the mixed-precision refinement.  Pinned with exact small-integer data. */
void or_spmv_f32(i64 n, const i32* rowptr, const i32* col, const float* val,
                 const float* x, float* y) {
  for (i64 i = 0; i < n; ++i) {
    float s = 0.0f;
    for (i64 k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = s;
  }
}

static double dot(i64 n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (i64 i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}
static double nrm2(i64 n, const double* a) { return sqrt(dot(n, a, a)); }

/* r = b - A x */
static void residual(i64 n, const i32* rp, const i32* ci, const double* v,
                     const double* b, const double* x, double* r) {
  or_spmv(n, rp, ci, v, x, r);
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i) r[i] = b[i] - r[i];
}

/* ------------------------------------------------------------------------- */
/* Conjugate gradient (Hestenes-Stiefel).                                      */
/*   r0 = b - A x0, p0 = r0                                                    */
/*   alpha = (r,r)/(Ap,p); x += alpha p; r -= alpha Ap;                        */
/*   beta = (r+,r+)/(r,r); p = r+ + beta p                                     */
/* Stops when the recursively updated ||r|| <= tol ||b||; the true residual    */
/* b - A x is then recomputed, and if it is above tol the iteration restarts   */
/* from the current x (residual replacement).                                 */
/* Returns iterations (number of alpha steps).  status: 0 ok, 4 not converged, */
/* 5 breakdown ((Ap,p) <= 0 with r != 0, i.e. A not SPD).                      */
/* alpha/beta histories (for the Lanczos-Ritz pin) are written when non-NULL.  */
/* Pinned: A = I in one step; k distinct eigenvalues in k steps; Lanczos Ritz  */
/* values vs the closed-form Poisson spectrum; dense LU solution.              */
/* ------------------------------------------------------------------------- */
i64 or_cg(i64 n, const i32* rp, const i32* ci, const double* v,
          const double* b, double* x, double tol, i64 maxit,
          double* alpha_hist, double* beta_hist, i64 hist_cap,
          double* relres_true, i32* status) {
  double* r = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* ap = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  const double bnorm = nrm2(n, b);
  i64 it = 0;
  *status = 0;
  if (bnorm == 0.0) {
    for (i64 i = 0; i < n; ++i) x[i] = 0.0;
    *relres_true = 0.0;
    free(r); free(p); free(ap);
    return 0;
  }
  for (;;) {
    residual(n, rp, ci, v, b, x, r);
    double rr = dot(n, r, r);
    if (sqrt(rr) <= tol * bnorm) break;           /* true residual converged */
    if (it >= maxit) { *status = 4; break; }
    memcpy(p, r, sizeof(double) * n);
    int check = 0;  /* set when the recursive residual reaches tol */
    while (it < maxit) {
      or_spmv(n, rp, ci, v, p, ap);
      const double pap = dot(n, ap, p);
      if (!(pap > 0.0)) { *status = 5; break; }
      const double alpha = rr / pap;
#pragma omp parallel for schedule(static)
      for (i64 i = 0; i < n; ++i) x[i] += alpha * p[i];
#pragma omp parallel for schedule(static)
      for (i64 i = 0; i < n; ++i) r[i] -= alpha * ap[i];
      const double rr_new = dot(n, r, r);
      const double beta = rr_new / rr;
      if (alpha_hist && it < hist_cap) alpha_hist[it] = alpha;
      if (beta_hist && it < hist_cap) beta_hist[it] = beta;
      ++it;
      rr = rr_new;
      if (sqrt(rr) <= tol * bnorm) { check = 1; break; }
#pragma omp parallel for schedule(static)
      for (i64 i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    }
    if (*status == 5) break;
    if (!check) { /* maxit reached inside the loop */
      residual(n, rp, ci, v, b, x, r);
      if (nrm2(n, r) > tol * bnorm) *status = 4;
      break;
    }
  }
  residual(n, rp, ci, v, b, x, r);
  *relres_true = nrm2(n, r) / bnorm;
  free(r); free(p); free(ap);
  return it;
}

/* ------------------------------------------------------------------------- */
/* Restarted GMRES(m) with modified Gram-Schmidt and Givens rotations.         */
/*   cycle: r = b - A x, beta = ||r||, v1 = r / beta, g = beta e1             */
/*   for j = 1..m: w = A v_j; for i <= j: h_ij = (w, v_i), w -= h_ij v_i;     */
/*     h_{j+1,j} = ||w||; rotate column j by G_1..G_{j-1}; form G_j that      */
/*     zeroes h_{j+1,j}; g_{j+1} = -s_j g_j, g_j = c_j g_j;                    */
/*     stop the cycle when |g_{j+1}| <= tol ||b|| or h_{j+1,j} = 0;           */
/*     v_{j+1} = w / h_{j+1,j}                                                 */
/*   y = R^{-1} g (back substitution); x += V y; restart.                     */
/* Returns total inner steps.  res_hist[k] = |g_{j+1}| / ||b|| after step k    */
/* (the residual estimate, monotone within a cycle).                          */
/* Pinned: dense LU on small systems; finite termination with k distinct      */
/* eigenvalues; monotone cycle residual; GMRES <= CG residual on SPD.          */
/* ------------------------------------------------------------------------- */
i64 or_gmres(i64 n, const i32* rp, const i32* ci, const double* v,
             const double* b, double* x, double tol, i64 m, i64 maxit,
             double* res_hist, i64 hist_cap, double* relres_true, i32* status) {
  const i64 nn = n > 0 ? n : 1;
  double* V = (double*)malloc(sizeof(double) * nn * (m + 1));
  double* H = (double*)calloc((size_t)((m + 1) * m), sizeof(double)); /* H[i*m + j] */
  double* cs = (double*)malloc(sizeof(double) * m);
  double* sn = (double*)malloc(sizeof(double) * m);
  double* g = (double*)malloc(sizeof(double) * (m + 1));
  double* y = (double*)malloc(sizeof(double) * m);
  double* r = (double*)malloc(sizeof(double) * nn);
  const double bnorm = nrm2(n, b);
  i64 it = 0;
  *status = 0;
  if (bnorm == 0.0) {
    for (i64 i = 0; i < n; ++i) x[i] = 0.0;
    *relres_true = 0.0;
    goto done;
  }
  for (;;) {
    residual(n, rp, ci, v, b, x, r);
    const double beta = nrm2(n, r);
    if (beta <= tol * bnorm) break;
    if (it >= maxit) { *status = 4; break; }
    for (i64 i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (i64 i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    i64 j_done = 0;
    for (i64 j = 0; j < m && it < maxit; ++j) {
      double* w = V + (j + 1) * nn;
      or_spmv(n, rp, ci, v, V + j * nn, w);
      for (i64 i = 0; i <= j; ++i) {                 /* modified Gram-Schmidt */
        const double hij = dot(n, w, V + i * nn);
        H[i * m + j] = hij;
        for (i64 k = 0; k < n; ++k) w[k] -= hij * V[i * nn + k];
      }
      const double hn = nrm2(n, w);
      H[(j + 1) * m + j] = hn;
      for (i64 i = 0; i < j; ++i) {                  /* previous rotations */
        const double a = H[i * m + j], bb = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const double a = H[j * m + j], bb = H[(j + 1) * m + j];
      const double den = sqrt(a * a + bb * bb);
      cs[j] = (den == 0.0) ? 1.0 : a / den;
      sn[j] = (den == 0.0) ? 0.0 : bb / den;
      H[j * m + j] = cs[j] * a + sn[j] * bb;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (res_hist && it < hist_cap) res_hist[it] = fabs(g[j + 1]) / bnorm;
      ++it;
      j_done = j + 1;
      if (fabs(g[j + 1]) <= tol * bnorm || hn == 0.0) break;
      for (i64 k = 0; k < n; ++k) w[k] /= hn;
    }
    for (i64 i = j_done - 1; i >= 0; --i) {          /* back substitution */
      double s = g[i];
      for (i64 k = i + 1; k < j_done; ++k) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    for (i64 i = 0; i < j_done; ++i)
      for (i64 k = 0; k < n; ++k) x[k] += y[i] * V[i * nn + k];
  }
  residual(n, rp, ci, v, b, x, r);
  *relres_true = nrm2(n, r) / bnorm;
done:
  free(V); free(H); free(cs); free(sn); free(g); free(y); free(r);
  return it;
}

/* ------------------------------------------------------------------------- */
/* FP32 CG / GMRES for the inner solves of iterative refinement.  All vector   */
/* arithmetic is in float; stops at ||r|| <= tol ||b|| on the recursive (CG)   */
/* or estimated (GMRES) residual, no true-residual check (the outer FP64 loop  */
/* does that).  Returns steps taken.                                           */
/* ------------------------------------------------------------------------- */
static float fdot(i64 n, const float* a, const float* b) {
  float s = 0.0f;
  for (i64 i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static i64 cg_f32(i64 n, const i32* rp, const i32* ci, const float* v,
                  const float* b, float* x, float tol, i64 maxit) {
  float* r = (float*)malloc(sizeof(float) * n);
  float* p = (float*)malloc(sizeof(float) * n);
  float* ap = (float*)malloc(sizeof(float) * n);
  for (i64 i = 0; i < n; ++i) { x[i] = 0.0f; r[i] = b[i]; p[i] = b[i]; }
  float rr = fdot(n, r, r);
  const float stop = tol * sqrtf(rr);
  i64 it = 0;
  while (it < maxit && sqrtf(rr) > stop) {
    or_spmv_f32(n, rp, ci, v, p, ap);
    const float pap = fdot(n, ap, p);
    if (!(pap > 0.0f)) break;
    const float alpha = rr / pap;
    for (i64 i = 0; i < n; ++i) x[i] += alpha * p[i];
    for (i64 i = 0; i < n; ++i) r[i] -= alpha * ap[i];
    const float rr_new = fdot(n, r, r);
    const float beta = rr_new / rr;
    rr = rr_new;
    for (i64 i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    ++it;
  }
  free(r); free(p); free(ap);
  return it;
}

static i64 gmres_f32(i64 n, const i32* rp, const i32* ci, const float* v,
                     const float* b, float* x, float tol, i64 m, i64 maxit) {
  float* V = (float*)malloc(sizeof(float) * n * (m + 1));
  float* H = (float*)calloc((size_t)((m + 1) * m), sizeof(float));
  float* cs = (float*)malloc(sizeof(float) * m);
  float* sn = (float*)malloc(sizeof(float) * m);
  float* g = (float*)malloc(sizeof(float) * (m + 1));
  float* y = (float*)malloc(sizeof(float) * m);
  float* r = (float*)malloc(sizeof(float) * n);
  for (i64 i = 0; i < n; ++i) x[i] = 0.0f;
  const float bnorm = sqrtf(fdot(n, b, b));
  i64 it = 0;
  while (it < maxit) {
    or_spmv_f32(n, rp, ci, v, x, r);
    for (i64 i = 0; i < n; ++i) r[i] = b[i] - r[i];
    const float beta = sqrtf(fdot(n, r, r));
    if (beta <= tol * bnorm) break;
    for (i64 i = 0; i < n; ++i) V[i] = r[i] / beta;
    for (i64 i = 0; i <= m; ++i) g[i] = 0.0f;
    g[0] = beta;
    i64 jd = 0;
    for (i64 j = 0; j < m && it < maxit; ++j) {
      float* w = V + (j + 1) * n;
      or_spmv_f32(n, rp, ci, v, V + j * n, w);
      for (i64 i = 0; i <= j; ++i) {
        const float h = fdot(n, w, V + i * n);
        H[i * m + j] = h;
        for (i64 k = 0; k < n; ++k) w[k] -= h * V[i * n + k];
      }
      const float hn = sqrtf(fdot(n, w, w));
      H[(j + 1) * m + j] = hn;
      for (i64 i = 0; i < j; ++i) {
        const float a = H[i * m + j], bb = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const float a = H[j * m + j], bb = H[(j + 1) * m + j];
      const float den = sqrtf(a * a + bb * bb);
      cs[j] = den == 0.0f ? 1.0f : a / den;
      sn[j] = den == 0.0f ? 0.0f : bb / den;
      H[j * m + j] = cs[j] * a + sn[j] * bb;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jd = j + 1;
      if (fabsf(g[j + 1]) <= tol * bnorm || hn == 0.0f) break;
      for (i64 k = 0; k < n; ++k) w[k] /= hn;
    }
    for (i64 i = jd - 1; i >= 0; --i) {
      float s = g[i];
      for (i64 k = i + 1; k < jd; ++k) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    for (i64 i = 0; i < jd; ++i)
      for (i64 k = 0; k < n; ++k) x[k] += y[i] * V[i * n + k];
    if (jd > 0 && fabsf(g[jd]) <= tol * bnorm) break;
  }
  free(V); free(H); free(cs); free(sn); free(g); free(y); free(r);
  return it;
}

/* ------------------------------------------------------------------------- */
/* Mixed-precision iterative refinement.  x0 = 0.  Loop: r = b - A x in FP64;  */
/* stop when ||r|| <= tol ||b||; otherwise round A and r to FP32 (RN-even),    */
/* solve A d = r in FP32 with CG (solver = 0) or GMRES(m) (solver = 1) to     */
/* relative max(inner_tol, theta tol ||b|| / ||r||), then x += (double) d.     */
/* (theta = 0: every inner solve to inner_tol.  theta > 0: an inner solve     */
/* stops once its residual is theta tol ||b||, which is all the outer target  */
/* needs of the correction.)                                                   */
/* Returns outer iterations; *inner_total = inner steps summed.                */
/* Pinned: the final FP64 true residual, recomputed by the definition SpMV.    */
/* ------------------------------------------------------------------------- */
i64 or_ir_solve(i64 n, const i32* rp, const i32* ci, const double* v,
                const double* b, double* x, i32 solver, i64 m, double tol,
                double inner_tol, double theta, i64 max_outer, i64 max_inner,
                i64* inner_total, double* relres_true, i32* status) {
  i64 nnz = rp[n];
  float* v32 = (float*)malloc(sizeof(float) * (nnz > 0 ? nnz : 1));
  float* r32 = (float*)malloc(sizeof(float) * (n > 0 ? n : 1));
  float* d32 = (float*)malloc(sizeof(float) * (n > 0 ? n : 1));
  double* r = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  for (i64 k = 0; k < nnz; ++k) v32[k] = (float)v[k];
  for (i64 i = 0; i < n; ++i) x[i] = 0.0;
  const double bnorm = nrm2(n, b);
  i64 outer = 0;
  *inner_total = 0;
  *status = 0;
  if (bnorm == 0.0) { *relres_true = 0.0; goto done; }
  for (;;) {
    residual(n, rp, ci, v, b, x, r);
    const double rn = nrm2(n, r);
    *relres_true = rn / bnorm;
    if (rn <= tol * bnorm) break;
    if (outer >= max_outer) { *status = 4; break; }
    for (i64 i = 0; i < n; ++i) r32[i] = (float)r[i];
    double itol = inner_tol;
    if (theta * tol * bnorm / rn > itol) itol = theta * tol * bnorm / rn;
    i64 steps = solver == 0
        ? cg_f32(n, rp, ci, v32, r32, d32, (float)itol, max_inner)
        : gmres_f32(n, rp, ci, v32, r32, d32, (float)itol, m, max_inner);
    *inner_total += steps;
    for (i64 i = 0; i < n; ++i) x[i] += (double)d32[i];
    ++outer;
  }
done:
  free(v32); free(r32); free(d32); free(r);
  return outer;
}

/* ------------------------------------------------------------------------- */
/* The 15 features of Table IV, in table order:                                */
/*  0 nrows 1 ncols 2 nnz 3 density 4 mean 5 sd 6 cov 7 max 8 min 9 maxavg   */
/*  10 distavg 11 clusteravg 12 fill 13 ndiag 14 diagfill                      */
/* Readings where the table is incomplete:                                     */
/*  - sd is the population standard deviation (1/nrows), summed in row order. */
/*  - cov is the coefficient of variation sd/mean (0 when mean = 0).          */
/*  - distavg = (1/nrows) sum_i (c_i^last - c_i^first); empty rows add 0.      */
/*  - cl_i = longest run of consecutive column indices (step +1) in row i;     */
/*    an empty row has cl_i = 0.                                               */
/*  - fill = nrows*max/nnz, diagfill = nrows*ndiag/nnz (0 when nnz = 0).       */
/*  - ndiag = number of distinct (col - row) offsets present.                 */
/* Pinned: closed forms on Poisson 2D/3D, identity and dense; brute force.    */
/* ------------------------------------------------------------------------- */
void or_features(i64 nrows, i64 ncols, const i32* rp, const i32* ci,
                 double* f) {
  const i64 nnz = nrows > 0 ? rp[nrows] : 0;
  for (int k = 0; k < 15; ++k) f[k] = 0.0;
  f[0] = (double)nrows;
  f[1] = (double)ncols;
  f[2] = (double)nnz;
  if (nrows == 0) return;
  f[3] = (ncols > 0) ? (double)nnz / ((double)nrows * (double)ncols) : 0.0;
  double sum_r = 0.0;
  i64 mx = 0, mn = -1;
  for (i64 i = 0; i < nrows; ++i) {
    const i64 r = rp[i + 1] - rp[i];
    sum_r += (double)r;
    if (r > mx) mx = r;
    if (mn < 0 || r < mn) mn = r;
  }
  const double mean = sum_r / (double)nrows;
  double ss = 0.0;
  for (i64 i = 0; i < nrows; ++i) {
    const double d = mean - (double)(rp[i + 1] - rp[i]);
    ss += d * d;
  }
  const double sd = sqrt(ss / (double)nrows);
  f[4] = mean;
  f[5] = sd;
  f[6] = mean != 0.0 ? sd / mean : 0.0;
  f[7] = (double)mx;
  f[8] = (double)mn;
  f[9] = (double)mx - mean;
  double dist = 0.0, clus = 0.0;
  for (i64 i = 0; i < nrows; ++i) {
    const i64 s = rp[i], e = rp[i + 1];
    if (e == s) continue;
    dist += (double)(ci[e - 1] - ci[s]);
    i64 best = 1, run = 1;
    for (i64 k = s + 1; k < e; ++k) {
      run = (ci[k] == ci[k - 1] + 1) ? run + 1 : 1;
      if (run > best) best = run;
    }
    clus += (double)best;
  }
  f[10] = dist / (double)nrows;
  f[11] = clus / (double)nrows;
  /* ndiag: mark every offset col - row (shifted by nrows - 1) in a byte map */
  const i64 span = nrows + ncols - 1;
  unsigned char* seen = (unsigned char*)calloc((size_t)(span > 0 ? span : 1), 1);
  i64 ndiag = 0;
  for (i64 i = 0; i < nrows; ++i)
    for (i64 k = rp[i]; k < rp[i + 1]; ++k) {
      const i64 off = (i64)ci[k] - i + (nrows - 1);
      if (!seen[off]) { seen[off] = 1; ++ndiag; }
    }
  free(seen);
  f[13] = (double)ndiag;
  if (nnz > 0) {
    f[12] = (double)nrows * (double)mx / (double)nnz;
    f[14] = (double)nrows * (double)ndiag / (double)nnz;
  }
}

/* ------------------------------------------------------------------------- */
/* Canonical format layouts.  All conversions copy indices and values bit for  */
/* bit.  Pinned: hand-derived layouts of a small matrix and round trips.       */
/* ------------------------------------------------------------------------- */

/* COO: entries in CSR (row-major) order. */
void or_csr_to_coo(i64 n, const i32* rp, const i32* ci, const double* v,
                   i32* row, i32* col, double* val) {
  for (i64 i = 0; i < n; ++i)
    for (i64 k = rp[i]; k < rp[i + 1]; ++k) {
      row[k] = (i32)i; col[k] = ci[k]; val[k] = v[k];
    }
}

/* COO (row-major sorted) back to CSR. */
void or_coo_to_csr(i64 n, i64 nnz, const i32* row, const i32* col,
                   const double* val, i32* rp, i32* ci, double* v) {
  for (i64 i = 0; i <= n; ++i) rp[i] = 0;
  for (i64 k = 0; k < nnz; ++k) rp[row[k] + 1]++;
  for (i64 i = 0; i < n; ++i) rp[i + 1] += rp[i];
  for (i64 k = 0; k < nnz; ++k) { ci[k] = col[k]; v[k] = val[k]; }
}

/* ELL: width K (>= the longest row), leading dimension ld (>= n), column-major:
 * entry k of row i at k*ld + i; padding has col = -1 and val = 0.0, including
 * the rows i in [n, ld). */
void or_csr_to_ell(i64 n, const i32* rp, const i32* ci, const double* v,
                   i64 K, i64 ld, i32* ecol, double* eval) {
  for (i64 k = 0; k < K; ++k)
    for (i64 i = 0; i < ld; ++i) {
      const i64 len = (i < n) ? rp[i + 1] - rp[i] : 0;
      if (k < len) { ecol[k * ld + i] = ci[rp[i] + k]; eval[k * ld + i] = v[rp[i] + k]; }
      else { ecol[k * ld + i] = -1; eval[k * ld + i] = 0.0; }
    }
}

/* ELL back to CSR (drops padding, which sits after a row's entries). */
void or_ell_to_csr(i64 n, i64 K, i64 ld, const i32* ecol, const double* eval,
                   i32* rp, i32* ci, double* v) {
  i64 pos = 0;
  rp[0] = 0;
  for (i64 i = 0; i < n; ++i) {
    for (i64 k = 0; k < K; ++k) {
      if (ecol[k * ld + i] < 0) break;
      ci[pos] = ecol[k * ld + i]; v[pos] = eval[k * ld + i]; ++pos;
    }
    rp[i + 1] = (i32)pos;
  }
}

/* SELL-C-sigma.  Rows are taken in windows of sigma consecutive rows; inside a
 * window they are ordered by length, longest first, ties kept in original
 * order (stable).  perm[s] = original row at sorted position s (length n).
 * Chunk c holds sorted positions [cC, cC + C); its width chunk_len[c] is the
 * longest row in it; positions >= n count as empty rows.  chunk_ptr[c] is the
 * offset of chunk c in col/val; chunk_ptr[c+1] = chunk_ptr[c] + C*chunk_len[c].
 * Entry k of slot r of chunk c is at chunk_ptr[c] + k*C + r; padding has
 * col = -1, val = 0.0.
 * or_sell_sizes fills perm, chunk_len, chunk_ptr (nchunks = ceil(n / C)) and
 * returns the total number of slots chunk_ptr[nchunks]. */
i64 or_sell_sizes(i64 n, const i32* rp, i64 C, i64 sigma, i32* perm,
                  i32* chunk_len, i64* chunk_ptr) {
  for (i64 w0 = 0; w0 < n; w0 += sigma) {
    const i64 w1 = (w0 + sigma < n) ? w0 + sigma : n;
    /* stable insertion sort of the window by descending length */
    for (i64 i = w0; i < w1; ++i) {
      const i32 row = (i32)i;
      const i64 len = rp[i + 1] - rp[i];
      i64 j = i;
      while (j > w0 && (rp[perm[j - 1] + 1] - rp[perm[j - 1]]) < len) {
        perm[j] = perm[j - 1];
        --j;
      }
      perm[j] = row;
    }
  }
  const i64 nchunks = (n + C - 1) / C;
  chunk_ptr[0] = 0;
  for (i64 c = 0; c < nchunks; ++c) {
    i64 w = 0;
    for (i64 r = 0; r < C; ++r) {
      const i64 s = c * C + r;
      if (s >= n) break;
      const i64 len = rp[perm[s] + 1] - rp[perm[s]];
      if (len > w) w = len;
    }
    chunk_len[c] = (i32)w;
    chunk_ptr[c + 1] = chunk_ptr[c] + C * w;
  }
  return chunk_ptr[nchunks];
}

void or_csr_to_sell(i64 n, const i32* rp, const i32* ci, const double* v,
                    i64 C, const i32* perm, const i32* chunk_len,
                    const i64* chunk_ptr, i32* scol, double* sval) {
  const i64 nchunks = (n + C - 1) / C;
  for (i64 c = 0; c < nchunks; ++c)
    for (i64 k = 0; k < chunk_len[c]; ++k)
      for (i64 r = 0; r < C; ++r) {
        const i64 s = c * C + r;
        const i64 at = chunk_ptr[c] + k * C + r;
        const i64 len = (s < n) ? rp[perm[s] + 1] - rp[perm[s]] : 0;
        if (k < len) { scol[at] = ci[rp[perm[s]] + k]; sval[at] = v[rp[perm[s]] + k]; }
        else { scol[at] = -1; sval[at] = 0.0; }
      }
}

void or_sell_to_csr(i64 n, i64 C, const i32* perm, const i32* chunk_len,
                    const i64* chunk_ptr, const i32* scol, const double* sval,
                    i32* rp, i32* ci, double* v) {
  /* row lengths first, then the entries of each original row */
  i32* len = (i32*)calloc((size_t)(n > 0 ? n : 1), sizeof(i32));
  for (i64 s = 0; s < n; ++s) {
    const i64 c = s / C, r = s % C;
    i32 l = 0;
    for (i64 k = 0; k < chunk_len[c]; ++k) {
      if (scol[chunk_ptr[c] + k * C + r] < 0) break;
      ++l;
    }
    len[perm[s]] = l;
  }
  rp[0] = 0;
  for (i64 i = 0; i < n; ++i) rp[i + 1] = rp[i] + len[i];
  for (i64 s = 0; s < n; ++s) {
    const i64 c = s / C, r = s % C;
    const i32 row = perm[s];
    for (i64 k = 0; k < len[row]; ++k) {
      ci[rp[row] + k] = scol[chunk_ptr[c] + k * C + r];
      v[rp[row] + k] = sval[chunk_ptr[c] + k * C + r];
    }
  }
  free(len);
}

/* HYB: an ELL part of width K (the first min(len, K) entries of every row,
 * same layout as or_csr_to_ell) plus a COO part holding the remaining entries
 * in row-major order.  Returns the COO entry count; with coo arrays NULL it
 * only counts. */
i64 or_csr_to_hyb(i64 n, const i32* rp, const i32* ci, const double* v,
                  i64 K, i64 ld, i32* ecol, double* eval, i32* crow,
                  i32* ccol, double* cval) {
  i64 nc = 0;
  for (i64 i = 0; i < n; ++i) {
    const i64 len = rp[i + 1] - rp[i];
    for (i64 k = K; k < len; ++k) {
      if (crow) { crow[nc] = (i32)i; ccol[nc] = ci[rp[i] + k]; cval[nc] = v[rp[i] + k]; }
      ++nc;
    }
  }
  if (ecol) {
    for (i64 k = 0; k < K; ++k)
      for (i64 i = 0; i < ld; ++i) {
        const i64 len = (i < n) ? rp[i + 1] - rp[i] : 0;
        if (k < len) { ecol[k * ld + i] = ci[rp[i] + k]; eval[k * ld + i] = v[rp[i] + k]; }
        else { ecol[k * ld + i] = -1; eval[k * ld + i] = 0.0; }
      }
  }
  return nc;
}

void or_hyb_to_csr(i64 n, i64 K, i64 ld, const i32* ecol, const double* eval,
                   i64 ncoo, const i32* crow, const i32* ccol,
                   const double* cval, i32* rp, i32* ci, double* v) {
  i64 pos = 0, q = 0;
  rp[0] = 0;
  for (i64 i = 0; i < n; ++i) {
    for (i64 k = 0; k < K; ++k) {
      if (ecol[k * ld + i] < 0) break;
      ci[pos] = ecol[k * ld + i]; v[pos] = eval[k * ld + i]; ++pos;
    }
    while (q < ncoo && crow[q] == i) { ci[pos] = ccol[q]; v[pos] = cval[q]; ++pos; ++q; }
    rp[i + 1] = (i32)pos;
  }
}

/* DIA: the distinct diagonal offsets (col - row) in ascending order, and a
 * value array of ndiag columns of nrows entries: entry of row i on diagonal d
 * at d*nrows + i, 0.0 where the diagonal has no entry in that row (including
 * positions outside the matrix).  or_dia_offsets fills offs (capacity
 * nrows + ncols - 1) and returns ndiag. */
i64 or_dia_offsets(i64 n, i64 ncols, const i32* rp, const i32* ci, i32* offs) {
  const i64 span = n + ncols - 1;
  unsigned char* seen = (unsigned char*)calloc((size_t)(span > 0 ? span : 1), 1);
  for (i64 i = 0; i < n; ++i)
    for (i64 k = rp[i]; k < rp[i + 1]; ++k) seen[(i64)ci[k] - i + (n - 1)] = 1;
  i64 nd = 0;
  for (i64 o = 0; o < span; ++o)
    if (seen[o]) offs[nd++] = (i32)(o - (n - 1));
  free(seen);
  return nd;
}

void or_csr_to_dia(i64 n, const i32* rp, const i32* ci, const double* v, i64 ndiag,
                   const i32* offs, double* data) {
  for (i64 q = 0; q < ndiag * n; ++q) data[q] = 0.0;
  for (i64 i = 0; i < n; ++i)
    for (i64 k = rp[i]; k < rp[i + 1]; ++k) {
      const i64 off = (i64)ci[k] - i;
      i64 d = 0;
      while (offs[d] != off) ++d;  /* offsets are few; linear search */
      data[d * n + i] = v[k];
    }
}

/* ------------------------------------------------------------------------- */
/* Predictor MLP (FP64).  Layer sizes d -> h1 -> h2 -> k, ReLU after the two   */
/* hidden layers, softmax cross-entropy averaged over the batch.               */
/* Flat parameter layout: W1[h1][d], b1[h1], W2[h2][h1], b2[h2], W3[k][h2],    */
/* b3[k] (row-major, output index first).                                      */
/* Pinned: central finite differences of the loss.                             */
/* ------------------------------------------------------------------------- */
i64 or_mlp_nparams(i64 d, i64 h1, i64 h2, i64 k) {
  return h1 * d + h1 + h2 * h1 + h2 + k * h2 + k;
}

static void layer(i64 nin, i64 nout, const double* W, const double* bias,
                  const double* in, double* out, int relu) {
  for (i64 o = 0; o < nout; ++o) {
    double s = bias[o];
    for (i64 i = 0; i < nin; ++i) s += W[o * nin + i] * in[i];
    out[o] = (relu && s < 0.0) ? 0.0 : s;
  }
}

/* logits[N][k] for inputs X[N][d] */
void or_mlp_forward(i64 N, i64 d, i64 h1, i64 h2, i64 k, const double* P,
                    const double* X, double* logits) {
  const double *W1 = P, *b1 = W1 + h1 * d, *W2 = b1 + h1, *b2 = W2 + h2 * h1;
  const double *W3 = b2 + h2, *b3 = W3 + k * h2;
  double* a1 = (double*)malloc(sizeof(double) * h1);
  double* a2 = (double*)malloc(sizeof(double) * h2);
  for (i64 s = 0; s < N; ++s) {
    layer(d, h1, W1, b1, X + s * d, a1, 1);
    layer(h1, h2, W2, b2, a1, a2, 1);
    layer(h2, k, W3, b3, a2, logits + s * k, 0);
  }
  free(a1); free(a2);
}

/* Mean softmax cross-entropy over the batch and its gradient dP (same layout
 * as P).  Returns the loss. */
double or_mlp_loss_grad(i64 N, i64 d, i64 h1, i64 h2, i64 k, const double* P,
                        const double* X, const i32* label, double* dP) {
  const double *W1 = P, *b1 = W1 + h1 * d, *W2 = b1 + h1, *b2 = W2 + h2 * h1;
  const double *W3 = b2 + h2, *b3 = W3 + k * h2;
  const i64 np = or_mlp_nparams(d, h1, h2, k);
  double *dW1 = dP, *db1 = dW1 + h1 * d, *dW2 = db1 + h1, *db2 = dW2 + h2 * h1;
  double *dW3 = db2 + h2, *db3 = dW3 + k * h2;
  for (i64 i = 0; i < np; ++i) dP[i] = 0.0;
  double* a1 = (double*)malloc(sizeof(double) * h1);
  double* a2 = (double*)malloc(sizeof(double) * h2);
  double* z = (double*)malloc(sizeof(double) * k);
  double* g3 = (double*)malloc(sizeof(double) * k);
  double* g2 = (double*)malloc(sizeof(double) * h2);
  double* g1 = (double*)malloc(sizeof(double) * h1);
  double loss = 0.0;
  for (i64 s = 0; s < N; ++s) {
    const double* x = X + s * d;
    layer(d, h1, W1, b1, x, a1, 1);
    layer(h1, h2, W2, b2, a1, a2, 1);
    layer(h2, k, W3, b3, a2, z, 0);
    double zmax = z[0];
    for (i64 o = 1; o < k; ++o) if (z[o] > zmax) zmax = z[o];
    double se = 0.0;
    for (i64 o = 0; o < k; ++o) se += exp(z[o] - zmax);
    const double lse = zmax + log(se);
    loss += lse - z[label[s]];
    /* dL/dz = softmax(z) - onehot, scaled by 1/N */
    for (i64 o = 0; o < k; ++o)
      g3[o] = (exp(z[o] - lse) - (o == label[s] ? 1.0 : 0.0)) / (double)N;
    for (i64 o = 0; o < k; ++o) {
      db3[o] += g3[o];
      for (i64 i = 0; i < h2; ++i) dW3[o * h2 + i] += g3[o] * a2[i];
    }
    for (i64 i = 0; i < h2; ++i) {
      double s2 = 0.0;
      for (i64 o = 0; o < k; ++o) s2 += W3[o * h2 + i] * g3[o];
      g2[i] = a2[i] > 0.0 ? s2 : 0.0;
    }
    for (i64 o = 0; o < h2; ++o) {
      db2[o] += g2[o];
      for (i64 i = 0; i < h1; ++i) dW2[o * h1 + i] += g2[o] * a1[i];
    }
    for (i64 i = 0; i < h1; ++i) {
      double s1 = 0.0;
      for (i64 o = 0; o < h2; ++o) s1 += W2[o * h1 + i] * g2[o];
      g1[i] = a1[i] > 0.0 ? s1 : 0.0;
    }
    for (i64 o = 0; o < h1; ++o) {
      db1[o] += g1[o];
      for (i64 i = 0; i < d; ++i) dW1[o * d + i] += g1[o] * x[i];
    }
  }
  free(a1); free(a2); free(z); free(g3); free(g2); free(g1);
  return loss / (double)N;
}

/* Mean cross-entropy with soft targets: for sample s with logits z and target
 * distribution q = Q[s][0..k) (rows >= 0 summing to 1), the loss is
 * logsumexp(z) - sum_c q_c z_c, and its gradient in z is softmax(z) - q (the
 * one-hot q of a label gives or_mlp_loss_grad).  Returns the mean loss and the
 * gradient dP of that mean, in P's layout.  Pinned: central finite differences;
 * one-hot targets reproduce or_mlp_loss_grad; log k at zero weights for any q. */
double or_mlp_loss_grad_soft(i64 N, i64 d, i64 h1, i64 h2, i64 k, const double* P,
                             const double* X, const double* Q, double* dP) {
  const double *W1 = P, *b1 = W1 + h1 * d, *W2 = b1 + h1, *b2 = W2 + h2 * h1;
  const double *W3 = b2 + h2, *b3 = W3 + k * h2;
  const i64 np = or_mlp_nparams(d, h1, h2, k);
  double *dW1 = dP, *db1 = dW1 + h1 * d, *dW2 = db1 + h1, *db2 = dW2 + h2 * h1;
  double *dW3 = db2 + h2, *db3 = dW3 + k * h2;
  for (i64 i = 0; i < np; ++i) dP[i] = 0.0;
  double* a1 = (double*)malloc(sizeof(double) * h1);
  double* a2 = (double*)malloc(sizeof(double) * h2);
  double* z = (double*)malloc(sizeof(double) * k);
  double* g3 = (double*)malloc(sizeof(double) * k);
  double* g2 = (double*)malloc(sizeof(double) * h2);
  double* g1 = (double*)malloc(sizeof(double) * h1);
  double loss = 0.0;
  for (i64 s = 0; s < N; ++s) {
    const double* x = X + s * d;
    const double* q = Q + s * k;
    layer(d, h1, W1, b1, x, a1, 1);
    layer(h1, h2, W2, b2, a1, a2, 1);
    layer(h2, k, W3, b3, a2, z, 0);
    double zmax = z[0];
    for (i64 o = 1; o < k; ++o) if (z[o] > zmax) zmax = z[o];
    double se = 0.0;
    for (i64 o = 0; o < k; ++o) se += exp(z[o] - zmax);
    const double lse = zmax + log(se);
    double qz = 0.0;
    for (i64 o = 0; o < k; ++o) qz += q[o] * z[o];
    loss += lse - qz;
    /* dL/dz = softmax(z) - q, scaled by 1/N */
    for (i64 o = 0; o < k; ++o) g3[o] = (exp(z[o] - lse) - q[o]) / (double)N;
    for (i64 o = 0; o < k; ++o) {
      db3[o] += g3[o];
      for (i64 i = 0; i < h2; ++i) dW3[o * h2 + i] += g3[o] * a2[i];
    }
    for (i64 i = 0; i < h2; ++i) {
      double s2 = 0.0;
      for (i64 o = 0; o < k; ++o) s2 += W3[o * h2 + i] * g3[o];
      g2[i] = a2[i] > 0.0 ? s2 : 0.0;
    }
    for (i64 o = 0; o < h2; ++o) {
      db2[o] += g2[o];
      for (i64 i = 0; i < h1; ++i) dW2[o * h1 + i] += g2[o] * a1[i];
    }
    for (i64 i = 0; i < h1; ++i) {
      double s1 = 0.0;
      for (i64 o = 0; o < h2; ++o) s1 += W2[o * h1 + i] * g2[o];
      g1[i] = a1[i] > 0.0 ? s1 : 0.0;
    }
    for (i64 o = 0; o < h1; ++o) {
      db1[o] += g1[o];
      for (i64 i = 0; i < d; ++i) dW1[o * d + i] += g1[o] * x[i];
    }
  }
  free(a1); free(a2); free(z); free(g3); free(g2); free(g1);
  return loss / (double)N;
}

/* One Adam step (Kingma and Ba), step count t >= 1:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * P -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
void or_adam_step(i64 np, double* P, const double* G, double* m, double* v,
                  i64 t, double lr, double b1, double b2, double eps) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (i64 i = 0; i < np; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * G[i];
    v[i] = b2 * v[i] + (1.0 - b2) * G[i] * G[i];
    P[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}
