/*
 * cascade.h -- C ABI of libcascade: SpMV-based Krylov solvers with cascaded
 * SpMV-configuration prediction and asynchronous execution, for NVIDIA B300
 * (sm_103a).  Method: Gao et al., "Cascaded Prediction and Asynchronous
 * Execution of Iterative Algorithms on Heterogeneous Platforms" (arXiv
 * 2411.10143).
 *
 * Conventions for every entry point
 *  - Every function returns a cp_status and never aborts the process.  On an
 *    error, cp_last_error() returns a message for the calling thread.
 *  - Pointers documented as "device" must point to memory of the context's
 *    device (cudaMalloc, torch CUDA tensors); "host" pointers are ordinary
 *    (optionally pinned) host memory.  No entry point keeps a caller pointer
 *    after it returns unless stated.
 *  - Index arrays are int32 (nnz <= 2^31 - 1 is checked); values are IEEE
 *    binary64 unless a dtype argument says binary32.
 *  - Work is issued on the context's main stream (and, for prediction, its
 *    side stream).  Entry points that return results to the host synchronise
 *    the streams they used before returning; cp_spmv does not (it is ordered on
 *    the main stream like a library kernel call).
 *  - A cp_ctx and the cp_mat objects created from it may be used by one host
 *    thread at a time.
 */
#ifndef CASCADE_H
#define CASCADE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cp_ctx cp_ctx;
typedef struct cp_mat cp_mat;

typedef enum {
  CP_OK = 0,
  CP_ERR_INVALID = 1,        /* bad argument or malformed CSR                      */
  CP_ERR_OOM = 2,            /* device allocation failed                           */
  CP_ERR_FOOTPRINT = 3,      /* a padded format would exceed its memory budget     */
  CP_ERR_NOT_CONVERGED = 4,  /* maxit reached; x holds the last iterate            */
  CP_ERR_BREAKDOWN = 5,      /* (Ap,p) <= 0 in CG, or a NaN/Inf appeared           */
  CP_ERR_TIMEOUT = 6,        /* a bounded wait gave up                             */
  CP_ERR_CUDA = 7,           /* a CUDA runtime call failed                         */
  CP_ERR_CANCELLED = 8,      /* work cancelled before it finished                  */
  CP_ERR_UNSUPPORTED = 9     /* configuration outside the supported space          */
} cp_status;

/* ------------------------------------------------------------------ configs */
/* SpMV configuration space (Sec. III-B-2, Fig. 2): compression format, then the
 * SpMV algorithm for that format, then the kernel parameter.  The paper's space
 * is COO/CSR/ELL/DIA/HYB across three libraries with the CSR-Vector threads per
 * vector (TpV) in {2,4,8,16,32}; this library's space is the formats below
 * (adding SELL-C-sigma, the slicing of Sec. V-A), the CSR algorithms scalar /
 * vector / merge-path, TpV for CSR-vector and the sort window sigma for SELL. */
enum {
  CP_FMT_CSR = 0,
  CP_FMT_COO = 1,
  CP_FMT_ELL = 2,
  CP_FMT_SELL = 3,
  CP_FMT_HYB = 4,
  CP_FMT_DIA = 5,
  CP_NUM_FMT = 6
};
enum { CP_ALGO_SCALAR = 0, CP_ALGO_VECTOR = 1, CP_ALGO_MERGE = 2, CP_NUM_ALGO = 3 };

typedef struct {
  int32_t fmt;        /* CP_FMT_*                                                     */
  int32_t algo;       /* CSR only: CP_ALGO_*                                          */
  int32_t tpv;        /* CSR-vector threads per row: 2, 4, 8, 16 or 32                */
  int32_t sell_c;     /* SELL chunk height; only 32 is supported (one warp per chunk) */
  int32_t sell_sigma; /* SELL sort window: 1 (no sort) or a multiple of 32, <= 8192   */
  int32_t hyb_k;      /* HYB ELL width; 0 = the 75th percentile of the row lengths (at
                          least 1; ceil(mean row length) if that is 1,023 or more)      */
} cp_config;

/* The default configuration every solve starts from: CSR, scalar kernel (one
 * thread per row).  (The paper's default is CUSP-COO, Sec. III-C-2.) */
void cp_config_default(cp_config* cfg);

/* ------------------------------------------------------------------ context */
/* cp_create: a context on CUDA device `device`.  main_stream / side_stream are
 * cudaStream_t handles owned by the caller (e.g. torch streams; pass
 * cudaStreamLegacy, (void*)1, for the legacy default stream) or NULL, in which
 * case the context creates (and later destroys) non-blocking streams of its
 * own.  Inputs written on another stream must be complete (or ordered before
 * the call) when an entry point reads them.  The side stream runs feature
 * extraction, prediction and format conversion concurrently with the solve
 * (Sec. III-C-2).
 * Errors: CP_ERR_INVALID (bad device), CP_ERR_CUDA, CP_ERR_OOM. */
cp_status cp_create(cp_ctx** out, int32_t device, void* main_stream, void* side_stream);
/* cp_destroy: waits for the context's streams, stops its prediction side
 * thread (the second thread of Sec. III-C-2's asynchronous model), releases
 * its device memory pool, pinned buffers and the streams it created (streams
 * the caller passed stay the caller's).  Every cp_mat of the context must be
 * freed first.  NULL is accepted (no-op).  Errors: CP_ERR_CUDA. */
cp_status cp_destroy(cp_ctx* ctx);

/* Message describing the last error of the calling thread ("" if none). */
const char* cp_last_error(void);

/* Size in bytes of a public struct of this header, for bindings that mirror
 * them: which = 0 cp_config, 1 cp_solve_opts, 2 cp_solve_info, 3 cp_gate,
 * 4 cp_server_opts, 5 cp_request, 6 cp_result; -1 for any other value.  Host
 * only, needs no device. */
int64_t cp_abi_sizeof(int32_t which);

/* Number of kernels this context has launched since creation (all streams). */
cp_status cp_ctx_launch_count(cp_ctx* ctx, int64_t* count);

/* ------------------------------------------------------------------ matrices */
/* cp_csr_load: the online stage starts from a given iterative solver, sparse
 * matrix and default SpMV configuration (Sec. III-A, Fig. 3); this call hands
 * the matrix, in CSR (the default configuration's format), to the library.
 * It copies a CSR matrix into library-owned device memory and
 * validates it on the device (rowptr[0] = 0, rowptr non-decreasing,
 * rowptr[nrows] = nnz, 0 <= col < ncols, columns strictly increasing within
 * each row).  rowptr[nrows+1], col[nnz], val[nnz] are host pointers when
 * on_device = 0 and device pointers when on_device = 1; the caller keeps
 * ownership of them.  The returned handle owns the copy and every format later
 * converted from it.  nrows, ncols >= 1; nnz >= 0.
 * Errors: CP_ERR_INVALID (malformed matrix, sizes out of range), CP_ERR_OOM. */
cp_status cp_csr_load(cp_ctx* ctx, int64_t nrows, int64_t ncols, int64_t nnz,
                      const int32_t* rowptr, const int32_t* col, const double* val,
                      int32_t on_device, cp_mat** out);
/* cp_mat_free: releases the CSR copy and every converted format and cached
 * feature vector of `mat` (the storage a format change costs, Sec. III-C-1),
 * after the context's streams have finished with them.  NULL is accepted.
 * Errors: CP_ERR_CUDA. */
cp_status cp_mat_free(cp_mat* mat);

/* cp_mat_reset: drop every converted format and the cached features of `mat`,
 * returning it to the state cp_csr_load left (the CSR copy stays).  Used to
 * measure a solve's preprocessing (features, prediction, conversion) again. */
cp_status cp_mat_reset(cp_mat* mat);

/* Budget, in bytes, for one padded format (ELL, SELL, HYB's ELL part) of one
 * matrix; conversions above it fail with CP_ERR_FOOTPRINT.  Default: 4 GiB. */
cp_status cp_set_format_budget(cp_ctx* ctx, int64_t bytes);

/* ------------------------------------------------------------------ features */
/* cp_features: the 15 features of Table IV (Sec. III-B-1) computed on the GPU,
 * written to host array out[15] in table order: nrows, ncols, nnz, density,
 * mean, sd, cov, max, min, maxavg, distavg, clusteravg, fill, ndiag, diagfill.
 * Counts and sums are exact (int64); sd is the population standard deviation
 * from exact sums; cov = sd/mean; distavg = mean over rows of (last column -
 * first column), empty rows adding 0; clusteravg = mean over rows of the
 * longest run of consecutive columns; fill = nrows*max/nnz; ndiag = number of
 * distinct (col - row) offsets; diagfill = nrows*ndiag/nnz. */
cp_status cp_features(cp_ctx* ctx, cp_mat* mat, double* out15);

/* ------------------------------------------------------------------ formats */
/* cp_convert: materialise the format of `cfg` (CSR -> COO, ELL, SELL-C-sigma,
 * HYB or DIA) on the main stream and wait for it; the result is cached in `mat`.
 * Conversions copy indices and values bit for bit (Sec. III-C-1: a format
 * change needs storage and a conversion kernel).
 * Errors: CP_ERR_FOOTPRINT, CP_ERR_UNSUPPORTED, CP_ERR_OOM. */
cp_status cp_convert(cp_ctx* ctx, cp_mat* mat, const cp_config* cfg);

/* Arrays of a converted format, for inspection.  Layouts:
 *  COO : ROW[nnz] (COL and VAL are the CSR arrays), row-major order.
 *  ELL : ELL_COL / ELL_VAL [K*ld], entry k of row i at k*ld + i, ld = nrows
 *        rounded up to 32, padding col = -1, val = 0.0.  dims = {K, ld}.
 *  SELL: PERM[nrows] (original row at sorted position s), CHUNK_LEN[nchunks],
 *        CHUNK_PTR[nchunks+1] (int64), SELL_COL / SELL_VAL[slots]; rows sorted
 *        longest-first (stable) inside windows of sigma rows; entry k of slot r
 *        of chunk c at CHUNK_PTR[c] + k*C + r; padding col = -1, val = 0.0.
 *        dims = {nchunks, slots, C, sigma}.
 *  HYB : HYB_ELL_COL / HYB_ELL_VAL [K*ld] (first K entries per row, ELL layout)
 *        and HYB_COO_ROW / HYB_COO_COL / HYB_COO_VAL [ncoo] (the remaining
 *        entries, row-major).  dims = {K, ld, ncoo}.
 *  DIA : DIA_OFFSETS[ndiag] (int32, distinct col - row, ascending) and
 *        DIA_VAL[ndiag*nrows], entry of row i on diagonal d at d*nrows + i,
 *        0.0 where the diagonal has no entry.  dims = {ndiag, nrows}.  At most
 *        1024 diagonals; more fail with CP_ERR_FOOTPRINT.
 * cp_format_dims writes up to 4 int64 dims.  cp_format_export copies one array
 * to host memory dst (capacity bytes); *bytes receives its size. */
enum {
  CP_ARR_COO_ROW = 0,
  CP_ARR_ELL_COL = 1, CP_ARR_ELL_VAL = 2,
  CP_ARR_SELL_PERM = 3, CP_ARR_SELL_CHUNK_LEN = 4, CP_ARR_SELL_CHUNK_PTR = 5,
  CP_ARR_SELL_COL = 6, CP_ARR_SELL_VAL = 7,
  CP_ARR_HYB_ELL_COL = 8, CP_ARR_HYB_ELL_VAL = 9,
  CP_ARR_HYB_COO_ROW = 10, CP_ARR_HYB_COO_COL = 11, CP_ARR_HYB_COO_VAL = 12,
  CP_ARR_DIA_OFFSETS = 13, CP_ARR_DIA_VAL = 14
};
cp_status cp_format_dims(cp_ctx* ctx, cp_mat* mat, const cp_config* cfg, int64_t dims[4]);
cp_status cp_format_export(cp_ctx* ctx, cp_mat* mat, const cp_config* cfg, int32_t array_id,
                           void* dst, int64_t capacity, int64_t* bytes);

/* ------------------------------------------------------------------ SpMV */
/* cp_spmv: y = alpha * A x + beta * y with the kernel of `cfg` (NULL: the
 * default CSR-scalar kernel); converts the format first if needed (blocking).
 * dtype 0: x, y are FP64 device arrays; dtype 1: FP32 device arrays and the
 * matrix values rounded to FP32 (round-to-nearest-even).  x has ncols entries,
 * y has nrows.  When beta = 0, y is not read.  Ordered on the main stream; does
 * not synchronise.  SpMV dominates CG and GMRES time (Sec. I). */
enum { CP_DTYPE_F64 = 0, CP_DTYPE_F32 = 1 };
/* Errors: CP_ERR_INVALID, CP_ERR_FOOTPRINT, CP_ERR_UNSUPPORTED (conversion);
 * CP_ERR_TIMEOUT when an earlier merge-path SpMV on this matrix gave up a
 * bounded wait for its tile copies (that call's y was incomplete; the error is
 * reported once, at the matrix's next merge-path call). */
cp_status cp_spmv(cp_ctx* ctx, cp_mat* mat, const cp_config* cfg, int32_t dtype,
                  double alpha, const void* x, double beta, void* y);

/* cp_spmv_csr_merge_noalloc: y = A x with the merge-path CSR kernel, allocating
 * nothing.  The paper has no counterpart: this entry point exists for callers
 * that cannot call cudaMalloc at the point where they need an SpMV -- for
 * example code running inside a memory-pool or arena allocator that owns all
 * device memory, or a host callback where allocation would synchronise the
 * device -- and so can use neither a cp_ctx nor a cp_mat (both allocate).
 *  - rowptr[nrows+1], col[nnz], val[nnz] (FP64), x[ncols], y[nrows]: device
 *    pointers owned by the caller; the matrix must be a valid CSR (as
 *    cp_csr_load checks) -- this call does not validate it.
 *  - The kernel's scratch (one carry per tile of 1,792 merge items) is a fixed
 *    768 KiB file-scope device array that every GPU loading the library keeps
 *    until the process exits; nrows + nnz may be at most 117,440,512
 *    (65,536 tiles), larger inputs return CP_ERR_INVALID.
 *  - The first call on a device, with that device current, does a one-time
 *    set-up: it looks up that array's device address (cudaGetSymbolAddress),
 *    reads the SM count and sets the kernel's function attributes.  Make that
 *    first call before any stream capture; a call on a 1-row matrix with
 *    nnz = 0 (rowptr = {0, 0}, col and val may be NULL) is enough.
 *  - Work is queued on `stream` (a cudaStream_t, NULL = the default stream) of
 *    the current device; the call does not synchronise.  Every call shares the
 *    one scratch array, so calls that overlap on the GPU (other streams or
 *    other host threads) race and must be serialised by the caller.  Nothing in
 *    the scratch needs to start at zero: each call writes every carry it reads.
 * Errors: CP_ERR_INVALID (NULL pointer, sizes out of range or above the
 * maximum), CP_ERR_CUDA (launch failure). */
cp_status cp_spmv_csr_merge_noalloc(int64_t nrows, int64_t ncols, int64_t nnz,
                                    const int32_t* rowptr, const int32_t* col,
                                    const double* val, const double* x, double* y,
                                    void* stream);

/* ------------------------------------------------------------------ predictors */
/* Each cascade stage is a small MLP classifier d -> h1 -> h2 -> k (ReLU), fed
 * z_j = (log(1 + f_j) - mu_j) / sd_j of the 15 features (FP32).  Stages
 * (Sec. III-C-1, Fig. 5):
 *   CP_STAGE_FORMAT     k = 6: CSR, COO, ELL, SELL, HYB, DIA
 *   CP_STAGE_CSR_ALGO   k = 3: scalar, vector, merge      (used if FORMAT = CSR)
 *   CP_STAGE_CSR_TPV    k = 5: TpV 2, 4, 8, 16, 32        (used if ALGO = vector)
 *   CP_STAGE_SELL_SIGMA k = 4: sigma 1, 32, 1024, 8192    (used if FORMAT = SELL)
 * and one classifier outside the cascade, for the batched solve (the batching
 * pattern; the paper has no counterpart), trained on labels that the batching
 * autotuner (cp_batch_tune) measures:
 *   CP_STAGE_BATCH_TPR  k = 3: threads per row 1, 4, 16 of a system in
 *                       cp_batch_solve's kernel
 * Flat parameter layout (FP32): W1[h1][d], b1[h1], W2[h2][h1], b2[h2],
 * W3[k][h2], b3[k].  d = 15, h1, h2 <= 64. */
enum {
  CP_STAGE_FORMAT = 0, CP_STAGE_CSR_ALGO = 1, CP_STAGE_CSR_TPV = 2, CP_STAGE_SELL_SIGMA = 3,
  CP_STAGE_BATCH_TPR = 4, CP_NUM_STAGES = 5
};
/* Install the weights of one stage (host arrays, copied).  Without a model a
 * stage keeps the current choice (plain CSR is the fallback). */
cp_status cp_model_load(cp_ctx* ctx, int32_t stage, int32_t h1, int32_t h2, int32_t k,
                        const float* params, const float* mu, const float* sd);
/* Read back the current weights of a stage: dims = {d, h1, h2, k}; params
 * (capacity floats), mu[15], sd[15] are host arrays. */
cp_status cp_model_get(cp_ctx* ctx, int32_t stage, int32_t dims[4], float* params,
                       int64_t capacity, float* mu, float* sd);

/* Predictor kernels, exposed for training and for checking (device pointers,
 * FP32, main stream, no synchronisation):
 *  cp_mlp_forward  : logits[N][k] for inputs X[N][d].
 *  cp_mlp_loss_grad: mean softmax cross-entropy over the batch -> loss[1] and
 *                    its gradient grad[nparams] (same layout as params).
 *  cp_adam_step    : one Adam step (Kingma and Ba) on params with moments m, v
 *                    at step t >= 1.
 * scratch: device workspace of at least cp_mlp_scratch_floats(N, dims) floats. */
int64_t cp_mlp_nparams(int32_t d, int32_t h1, int32_t h2, int32_t k);
int64_t cp_mlp_scratch_floats(int64_t N, int32_t d, int32_t h1, int32_t h2, int32_t k);
cp_status cp_mlp_forward(cp_ctx* ctx, int64_t N, int32_t d, int32_t h1, int32_t h2, int32_t k,
                         const float* params, const float* X, float* logits, float* scratch);
cp_status cp_mlp_loss_grad(cp_ctx* ctx, int64_t N, int32_t d, int32_t h1, int32_t h2, int32_t k,
                           const float* params, const float* X, const int32_t* labels,
                           float* loss, float* grad, float* scratch);
cp_status cp_adam_step(cp_ctx* ctx, int64_t nparams, float* params, const float* grad, float* m,
                       float* v, int32_t t, float lr, float beta1, float beta2, float eps);
/* cp_mlp_loss_grad_soft: as cp_mlp_loss_grad with a target distribution per
 * sample instead of a class: targets[N][k] (device FP32, each row >= 0 and
 * summing to 1); loss = mean over the batch of logsumexp(z) - sum_c t_c z_c,
 * whose gradient in the logits is softmax(z) - t.  One-hot rows give
 * cp_mlp_loss_grad.  The cascade's labels come from measured SpMV times
 * (Sec. III-B-2); soft targets spread a sample's weight over the configurations
 * within a few percent of its fastest, so near-ties are learned as near-ties
 * and a costly mistake costs more than a cheap one. */
cp_status cp_mlp_loss_grad_soft(cp_ctx* ctx, int64_t N, int32_t d, int32_t h1, int32_t h2,
                                int32_t k, const float* params, const float* X,
                                const float* targets, float* loss, float* grad, float* scratch);

/* cp_model_train: train one stage on the GPU with the kernels above.  Host
 * inputs: raw features F[N][15] and labels[N] in [0, k); the standardisation
 * (mu, sd of log(1 + f)) is computed from F; weights are initialised from
 * `seed`; full-batch Adam for `epochs` steps with learning rate lr.  The
 * trained weights replace the stage's model.  final_loss (host, may be NULL)
 * receives the last loss.  (Sec. III-B-3 trains one classifier per stage.) */
cp_status cp_model_train(cp_ctx* ctx, int32_t stage, int64_t N, const double* F,
                         const int32_t* labels, int32_t h1, int32_t h2, int32_t k,
                         int32_t epochs, float lr, uint64_t seed, float* final_loss);
/* cp_model_train_soft: cp_model_train with host target distributions
 * targets[N][k] (FP32, rows >= 0 summing to 1 within 1e-4) in place of labels,
 * trained with cp_mlp_loss_grad_soft's loss.
 * Errors: CP_ERR_INVALID (a row that is not a distribution), CP_ERR_CUDA. */
cp_status cp_model_train_soft(cp_ctx* ctx, int32_t stage, int64_t N, const double* F,
                              const float* targets, int32_t h1, int32_t h2, int32_t k,
                              int32_t epochs, float lr, uint64_t seed, float* final_loss);

/* cp_predict_stage: one cascade stage's classifier (Sec. III-B-3: one trained
 * model per stage of Fig. 5's cascade) applied to a given feature vector, with
 * the kernel and the installed weights the cascade itself uses.
 *  - features15: host double[15], the Table IV features in cp_features order.
 *  - logits: host float[k] (k = the stage's classes, see the stage list above)
 *    or NULL; receives the stage's FP32 logits.
 *  - pick: host, may be NULL; receives the arg-max class (the first on ties),
 *    the choice the cascade takes at that stage.
 * Runs on the side stream and waits for it.  Exposed so that the inference
 * can be checked against a reference implementation of the classifier.
 * Errors: CP_ERR_INVALID (NULL features, bad stage, no model installed in the
 * stage), CP_ERR_CUDA. */
cp_status cp_predict_stage(cp_ctx* ctx, int32_t stage, const double* features15, float* logits,
                           int32_t* pick);

/* cp_predict: the sequential cascaded prediction (SerGMRES-style, Sec. IV-C):
 * features, then FORMAT, then the algorithm / parameter stage that applies,
 * on the side stream, joined before returning.  out receives the predicted
 * configuration; stage_ms (host float[4], may be NULL) receives the time of
 * feature extraction and of the three cascade steps. */
cp_status cp_predict(cp_ctx* ctx, cp_mat* mat, cp_config* out, float* stage_ms);

/* ------------------------------------------------------------------ solvers */
enum { CP_MODE_PLAIN = 0, CP_MODE_SEQUENTIAL = 1, CP_MODE_ASYNC = 2 };
enum { CP_PREC_FP64 = 0, CP_PREC_FP32_IR = 1 };

typedef struct {
  double tol;            /* relative residual ||b - Ax|| / ||b|| to reach (e.g. 1e-10)   */
  int32_t maxit;         /* iteration limit (SpMV steps; IR: inner steps in total)        */
  int32_t restart;       /* GMRES restart length m (e.g. 30), 1..64                      */
  int32_t mode;          /* PLAIN: default kernel throughout; SEQUENTIAL: predict, then
                            solve; ASYNC: solve at once on the default kernel while the
                            side stream predicts, switching kernel mid-run (Sec. III-C-2) */
  int32_t precision;     /* FP64, or FP32 inner solves inside FP64 iterative refinement   */
  double inner_tol;      /* FP32_IR: relative tolerance of each inner solve (e.g. 1e-5)  */
  int32_t max_outer;     /* FP32_IR: refinement steps limit                               */
  int32_t check_every;   /* iterations between host convergence checks (0: default 8)   */
  int32_t profile;       /* 1: time every SpMV launch with CUDA events (t_spmv_ms)        */
  int32_t iteration_kernel; /* CG and GMRES: 0 = one persistent cooperative launch runs
                            the iterations while the format has a persistent kernel
                            (CSR scalar / vector, ELL, SELL, DIA, HYB, COO; not
                            CSR-merge) and no prediction work is pending on the side stream,
                            falling back to one launch per step otherwise; 1 = always
                            one launch per step; 2 = alternate persistent launches of
                            persist_chunk iterations with as many one-launch-per-step
                            iterations (hands the iteration over between the two paths,
                            as a switch does, at every chunk; for tests)          */
  const cp_config* force;/* non-NULL: use this configuration from the first iteration    */
  double wait_limit_ms;  /* bound of every device-side wait of the persistent kernel (its
                            grid barriers); a wait that exceeds it ends the solve with
                            CP_ERR_TIMEOUT and the context stays usable.  0: 2000 ms    */
  int32_t persist_chunk; /* > 0: a persistent launch returns to the host after this many
                            iterations (the host launches again to go on), e.g. to poll
                            for cancellation; 0: it runs to the end of the solve      */
  int32_t gmres_orth;    /* persistent GMRES orthogonalisation: 0 = modified Gram-Schmidt
                            in groups of four columns where a block's rows of the new
                            vector fit in shared memory (n up to about 3 million rows
                            in FP64 at m = 30), else 1; 1 = classical Gram-Schmidt
                            with a second pass (conditional in FP64, always in FP32),
                            as the one-launch-per-step kernels use               */
  double ir_theta;       /* FP32_IR: an inner solve stops at relative inner_tol or as soon
                            as its residual is at most ir_theta * tol * ||b||, whichever
                            comes first: the correction need not be more accurate than
                            what the outer target asks.  In effect each inner solve runs
                            to relative max(inner_tol, ir_theta tol ||b|| / ||r_k||)
                            (r_k the outer residual).  0 = always to inner_tol; default
                            0.5; must be in [0, 1)                                  */
} cp_solve_opts;

typedef struct {
  int32_t iters;           /* SpMV steps of the Krylov iteration (all inner steps for IR) */
  int32_t outer_iters;     /* IR refinement steps (0 for FP64)                            */
  int32_t switch_iter[3];  /* iteration at which the FORMAT / ALGO / PARAM prediction was
                              applied, -1 if never (Table VII)                            */
  int32_t n_spmv;          /* SpMV launches timed when profile = 1                        */
  int32_t n_launches;      /* kernels launched by the solve                               */
  int32_t status;          /* the returned cp_status                                      */
  double relres_true;      /* ||b - A x|| / ||b|| recomputed in FP64 at exit              */
  cp_config final_cfg;     /* configuration in use at exit                                */
  float t_features_ms, t_predict_ms[3], t_convert_ms; /* side-stream step times           */
  float t_total_ms;        /* wall time from entry to x ready                             */
  float t_spmv_ms;         /* summed SpMV kernel time when profile = 1                    */
  float t_persist_ms;      /* summed duration of the persistent (CG or GMRES) launches    */
  int32_t persist_iters;   /* iterations those launches ran                               */
  float t_persist_last_ms; /* duration of the last persistent launch (final configuration) */
  int32_t persist_last_iters; /* iterations it ran                                        */
  int32_t gate_declined;   /* the cost-aware gate kept the default format (cp_gate): 1 after
                              the FORMAT stage, 2 before the feature pass (two-tier)      */
  float gate_remaining;    /* its estimate of the iterations left when it decided (-1: none) */
  float gate_cost_spmvs;   /* its estimate of the conversion cost, in default-kernel SpMVs */
  int32_t side_status;     /* the prediction side's first error (CP_OK if none): the solve
                              carries on with the configuration it has (the default CSR
                              kernel at worst) and still returns its own status          */
  int32_t persist_launches; /* persistent launches the solve made                           */
} cp_solve_info;

void cp_solve_opts_default(cp_solve_opts* opts);

/* ------------------------------------------------------------------ cost-aware switching
 * An extension of Sec. III-C-2's switch.  The paper converts whenever a
 * prediction lands.  Sec. II-B quotes conversion costs of 9 to 270 CSR SpMVs; in
 * Sec. IV-B the conversion outweighs the gain on a small matrix; Sec. V-C
 * describes selecting a format only when the iteration count, estimated from
 * the first iterations' residuals, is large enough.  Here, before converting to
 * the predicted format f, the side thread asks whether the
 * expected saving over the rest of the solve exceeds the conversion cost, in
 * units of one SpMV of the default kernel:
 *     remaining x (1 - 1/speedup[f])  >  cost_f(nnz)
 * remaining: iterations left, extrapolated from the residual decay the solve
 * has shown so far (geometric rate over the iterations done).  Krylov
 * residuals often fall fast at first, so a verdict to keep the default is
 * re-examined on later windows of 8, 16, ... iterations (at most 6) while the
 * estimate keeps growing by more than a quarter; a steady estimate is final;
 * speedup[f]: typical SpMV speedup of format f over the default kernel where
 * the classifier picks f; cost_f(nnz) = (conv_a_ms[f] + conv_b_ms[f] nnz/1e6) /
 * (spmv_a_ms + spmv_b_ms nnz/1e6), linear fits of conversion and default-SpMV
 * times.  All figures are measured on this GPU when the cascade is trained.
 * Indices of the arrays: CP_FMT_*. */
typedef struct {
  double speedup[6];
  double conv_a_ms[6], conv_b_ms[6];  /* conversion time = a + b * nnz / 1e6 (ms)       */
  double spmv_a_ms, spmv_b_ms;        /* default-kernel SpMV time = a + b * nnz / 1e6    */
  double feat_a_ms, feat_b_ms;        /* Table IV feature extraction time, same form     */
  int64_t small_rows;                 /* two-tier features below this many rows          */
  int32_t enabled;                    /* 0: always switch (the paper's behaviour)        */
} cp_gate;

/* cp_warmup: runs, once, every kernel a solve can launch -- features, the
 * cascade's inference when models are installed, each format's conversion and
 * SpMV in FP64 and FP32, CG and GMRES in both precisions on the persistent and
 * the per-step paths, and an asynchronous solve of each -- on a small internal
 * system (3D Poisson 10^3), so that no later solve pays the one-time cost of a
 * kernel's first launch in the process (the CUDA runtime loads kernels lazily;
 * measured: a first asynchronous GMRES(30) solve of 86 ms against 59 ms for the
 * next).  Takes about 0.1-0.3 s; the solves' time-to-solution (Sec. IV) assumes
 * it was made.  cp_server_create calls it.  Blocking; uses ctx's streams.
 * Errors: CP_ERR_CUDA, CP_ERR_OOM. */
cp_status cp_warmup(cp_ctx* ctx);

/* cp_fp64_fma_rate: measures this GPU's FP64 fused multiply-add rate (FMAs per
 * second, host double) with a kernel of independent FMA chains on every SM,
 * the best of five timed launches (CUDA events on the main stream).  The paper
 * has no counterpart: it is the denominator of the roofline of the kernels
 * bound by the FP64 pipe (persistent GMRES), measured rather than taken from a
 * data sheet.  Blocking; about 0.1 s.  Errors: CP_ERR_INVALID, CP_ERR_CUDA. */
cp_status cp_fp64_fma_rate(cp_ctx* ctx, double* fma_per_s);

/* Fault injection on the host, for tests of the asynchronous mode's recovery:
 * the next solve's prediction side thread raises an error at `point` (0: before
 * the feature pass, 1: after it, 2: after the FORMAT stage, before any
 * conversion; -1 cancels a pending injection).  One-shot.  Nothing runs on or
 * waits for the GPU differently; the solve must finish on the default kernel
 * and report the error in cp_solve_info.side_status. */
cp_status cp_inject_side_failure(cp_ctx* ctx, int32_t point);

/* Two-tier features (also an extension; Sec. II-B quotes Swann et al.: below
 * 100,000 rows, extracting the features costs more than one SpMV).  For a
 * matrix with fewer than small_rows rows, the side thread first applies the
 * rule with what costs O(1): the iterations left (from the residual decay),
 * the best speedup over all formats, and the cost of the O(nnz) feature pass
 * plus the cheapest conversion.  It computes the features (and runs the
 * cascade) only if even that best case pays.
 * Install (or, with enabled = 0, disable) the gate for solves in ctx. */
cp_status cp_gate_set(cp_ctx* ctx, const cp_gate* gate);
/* The gate's rule, on the host: 1 to convert and switch to format fmt, 0 to
 * keep the default.  fmt < 0: the first tier's rule (compute the features or
 * not), with the largest speedup[] and the feature pass plus the cheapest
 * conversion as the cost.  iters, res0, res: iterations done, the initial and the
 * latest residual norms; target: the residual norm that ends the solve
 * (tol * ||b||).  Too little history (iters < 2) or no decay yet counts as a
 * long solve (switch).  remaining and cost_spmvs (may be NULL) receive the
 * estimates (-1: unknown). */
int32_t cp_gate_decide(const cp_gate* gate, int32_t fmt, int64_t nnz, int32_t iters, double res0,
                       double res, double target, double* remaining, double* cost_spmvs);
/* The payback of the same rule (host only): the number of default-kernel
 * iterations after which a switch to format fmt has saved what its conversion
 * cost, cost_spmvs / (1 - 1/speedup) -- the break-even of cp_gate_decide's
 * "iterations left".  HUGE_VAL when no gain is expected (speedup <= 1); 0 when
 * the rule does not apply (gate NULL or disabled, fmt = 0 or >= 6).  fmt < 0 is
 * the first tier's best case.  When the payback is at most four iterations and
 * the solve is still more than 1e3 times above its target, the side thread
 * switches without waiting for the two iterations of residual history the rule
 * otherwise reads. */
double cp_gate_payback(const cp_gate* gate, int32_t fmt, int64_t nnz);

/* Speedups for the gate that follow the matrix.  speedup[f] of cp_gate is one
 * figure per format (the median over the training matrices labelled f), while a
 * format's gain varies with the matrix: on 3D stencils of about 10^5 rows SELL's
 * SpMV is 1.05x CSR-scalar's, against 1.16x for the SELL-labelled matrices, and
 * a switch made on the larger figure costs more than it saves.  With neighbours installed, the tier-one gate (features known) takes
 * for format f the median, over the k training matrices nearest to the matrix,
 * of their best measured SpMV speedup of f over the default kernel; the first
 * tier keeps cp_gate's figures.
 *
 * cp_gate_knn_speedup (host only): that estimate.  count training matrices:
 * z (count x 15 floats, row-major) their features standardised as the cascade's
 * inputs are, z = (log1p(f) - mu) / sd; speedup (count x 6 floats, CP_FMT_*
 * order, 0 where the format could not be built) their speedups.  features: the
 * matrix's 15 Table IV features.  Nearest by Euclidean distance in z, ties to
 * the lower index; the median of an even number of values is the mean of the
 * middle two.  k is clamped to count.  Writes *out; errors: CP_ERR_INVALID
 * (NULL pointer, count < 1, k < 1, fmt outside 0..5, sd <= 0). */
cp_status cp_gate_knn_speedup(int32_t count, int32_t k, const double* mu, const double* sd,
                              const float* z, const float* speedup, const double* features,
                              int32_t fmt, double* out);
/* Installs such neighbours in ctx (copied; count = 0 removes them, and the
 * gate uses cp_gate.speedup again).  Errors: CP_ERR_INVALID. */
cp_status cp_gate_set_neighbours(cp_ctx* ctx, int32_t count, int32_t k, const double* mu,
                                 const double* sd, const float* z, const float* speedup);

/* cp_solve_cg: CG (Sec. I) for SPD A.  b, x: device FP64 arrays of nrows
 * entries; x is read as x0 and overwritten with the solution.  info (host) may
 * be NULL.  Returns CP_OK when the true relative residual <= tol,
 * CP_ERR_NOT_CONVERGED (x = last iterate), CP_ERR_BREAKDOWN. */
cp_status cp_solve_cg(cp_ctx* ctx, cp_mat* mat, const double* b, double* x,
                      const cp_solve_opts* opts, cp_solve_info* info);

/* cp_solve_gmres: restarted GMRES(m) (Sec. IV-A) for nonsymmetric A; classical
 * Gram-Schmidt with one reorthogonalisation, Givens rotations and the
 * least-squares solve in FP64.  Arguments as cp_solve_cg. */
cp_status cp_solve_gmres(cp_ctx* ctx, cp_mat* mat, const double* b, double* x,
                         const cp_solve_opts* opts, cp_solve_info* info);

/* ------------------------------------------------------------------ batching */
/* cp_batch_solve: solve nsys small systems A_i x_i = b_i in one persistent
 * launch held in a CUDA graph (each context instantiates the graph of each
 * launch shape once and updates its kernel node per batch).  One thread block
 * per system at a time, systems taken from a device work queue, largest first
 * (or in the caller's order where the class's tuned schedule says so).
 * Every system runs FP64 iterative refinement to opts->tol around FP32 inner
 * solves to opts->inner_tol (stopping early as opts->ir_theta allows):
 * solver[i] = 0 for CG (SPD A_i), 1 for
 * GMRES(opts->restart), restart <= 32.  FP64 is kept for the outer residual,
 * the update of x and GMRES's Givens / least-squares step.  mats[i] (square,
 * CSR), b[i], x[i] (device FP64, x read as x0) are host arrays of nsys entries;
 * opts->maxit bounds the inner steps of each system.  The launch shape:
 *  - threads: threads per system, 128, 256, 512 or 1024; 0 = the schedule of
 *    the batch's class (the autotuner's choice, see cp_batch_tune, else a rule
 *    on the mean system size with a thread per row);
 *  - threads_per_row: 1 (CSR-scalar rows), 4 or 16 (groups of lanes share a
 *    row and add with shuffles, for long rows), for every system; 0 = each
 *    system its own: the CP_STAGE_BATCH_TPR classifier's pick for its matrix
 *    when that stage has a model (see cp_batch_tpr), else the class's
 *    schedule when threads = 0, else 1.
 * infos (host array of nsys, may be NULL) receives per-system iterations,
 * relres_true, status, and in t_total_ms the device time of the whole batched
 * launch (the same for every system).  Returns the first non-OK system status,
 * else CP_OK.
 * (The batching pattern; the paper's solver handles one system at a time.) */
cp_status cp_batch_solve(cp_ctx* ctx, int32_t nsys, cp_mat* const* mats, const int32_t* solver,
                         const double* const* b, double* const* x, const cp_solve_opts* opts,
                         int32_t threads, int32_t threads_per_row, cp_solve_info* infos);

/* cp_batch_tune: the batching autotuner (a systems addition for the batched
 * pattern; the paper has no counterpart).  Solves the given batch as
 * cp_batch_solve does, but into scratch solutions (the batch's own x are not
 * touched, x0 = 0), once per launch shape -- 128, 256, 512 and 1024 threads per
 * system, each with 1, 4 and 16 threads per row -- after one warm-up each,
 * timing each launch with CUDA events.  It records the fastest shape in a
 * per-device schedule under the batch's class: whether the batch holds a GMRES
 * system, and floor(log2(mean rows)).  The shapes are timed with the largest
 * systems dequeued first; the best shape is then timed once more with the
 * systems dequeued in the caller's order (the packing schedule), and the faster
 * order is recorded with it.  cp_batch_solve with threads = 0 then uses that
 * shape and order for batches of the class.  Arguments as cp_batch_solve.
 * best_threads / best_threads_per_row / best_order (may be NULL) receive the
 * choice (order 0: largest first, 1: the caller's order); ms (may be NULL, 12
 * floats) the times of the shapes, ms[3 t + r] for threads index t (128, 256,
 * 512, 1024) and threads-per-row index r (1, 4, 16); ms_order (may be NULL) the
 * best shape's time in the caller's order.  Any system that fails to converge
 * returns its status. */
cp_status cp_batch_tune(cp_ctx* ctx, int32_t nsys, cp_mat* const* mats, const int32_t* solver,
                        const double* const* b, const cp_solve_opts* opts,
                        int32_t* best_threads, int32_t* best_threads_per_row,
                        int32_t* best_order, float* ms, float* ms_order);
/* cp_batch_tpr: the threads per row cp_batch_solve(threads_per_row = 0) gives
 * the systems of matrix m when the CP_STAGE_BATCH_TPR stage has a model: the
 * classifier's pick on m's Table IV features (computed on the main stream if m
 * has none yet), kept with m for later batches.  *tpr (host int32) receives 1,
 * 4 or 16, or 0 when the stage has no model.  Synchronises the main stream the
 * first time for m.  Errors: CP_ERR_INVALID (NULL argument). */
cp_status cp_batch_tpr(cp_ctx* ctx, cp_mat* m, int32_t* tpr);
/* The launch shape cp_batch_solve(threads = 0) uses for a batch with mean_rows
 * rows per system (has_gmres: the batch holds a GMRES system): the tuned shape
 * and packing order of that class, else 128 / 256 / 512 / 1024 threads for mean
 * rows below 512 / 2048 / 8192 / above, with 1 thread per row, largest systems
 * first.  threads, threads_per_row, order (may be NULL; 0 largest first, 1 the
 * caller's order): host int32.  Errors: CP_ERR_INVALID (NULL argument). */
cp_status cp_batch_schedule(cp_ctx* ctx, int64_t mean_rows, int32_t has_gmres, int32_t* threads,
                            int32_t* threads_per_row, int32_t* order);

/* ------------------------------------------------------------------ serving */
/* A continuous-batching solve server.  Requests carry a matrix already loaded
 * with cp_csr_load (kept resident; several requests may share one), a device
 * right-hand side b and a device solution buffer x (x0 in, solution out), and
 * are admitted while their Krylov workspace fits mem_budget.  `lanes` worker
 * threads, each with its own streams, run admitted work concurrently: requests
 * with nrows <= small_max_n are packed into one persistent batched launch
 * (cp_batch_solve's kernel), larger ones run the full-GPU solver in `mode`
 * with FP32 inner solves inside FP64 refinement to tol.  Requests that arrive
 * while others run join as soon as a lane and memory free up.  The caller
 * keeps every request's buffers and matrix alive until its result is polled;
 * it must not free or reset a matrix while requests on it are in flight. */
typedef struct cp_server cp_server;
typedef struct {
  double tol;           /* relative residual per request (e.g. 1e-10)          */
  double inner_tol;     /* FP32 inner-solve tolerance (e.g. 1e-5)              */
  int32_t restart;      /* GMRES restart length, 1..32                          */
  int32_t maxit;        /* inner steps per request                              */
  int32_t small_max_n;  /* requests with nrows <= this are batched              */
  int32_t max_batch;    /* most requests in one batched launch                 */
  int32_t lanes;        /* concurrent jobs on the device, 1..32                 */
  int32_t mode;         /* CP_MODE_* of the full-GPU solver for large requests  */
  int64_t mem_budget;   /* bytes of solver workspace admitted at once           */
  int32_t small_max_n_gmres; /* GMRES requests are batched only up to this many rows
                           (<= small_max_n; default 8192): a batched system's
                           Krylov basis is streamed from HBM every step while
                           the batch's other systems share the bandwidth, so a
                           mid-size GMRES request is served faster by the
                           full-GPU persistent solver                          */
  double ir_theta;      /* inner-solve stop as cp_solve_opts.ir_theta (default 0.5) */
} cp_server_opts;
typedef struct {
  int64_t id;           /* caller's tag, returned in the result                 */
  cp_mat* mat;
  int32_t solver;       /* 0 CG, 1 GMRES                                         */
  int32_t reserved;
  const double* b;      /* device, nrows                                        */
  double* x;            /* device, nrows                                        */
} cp_request;
typedef struct {
  int64_t id;
  int32_t status, iters, batched, lane;
  double relres_true;
  double t_submit_ms, t_start_ms, t_done_ms;  /* since cp_server_create          */
} cp_result;

void cp_server_opts_default(cp_server_opts* opts);
/* The server uses the cascade models installed in ctx at creation time. */
cp_status cp_server_create(cp_ctx* ctx, const cp_server_opts* opts, cp_server** out);
cp_status cp_server_submit(cp_server* srv, const cp_request* req);
/* Move up to capacity finished results into out (host); *count receives how many. */
cp_status cp_server_poll(cp_server* srv, cp_result* out, int32_t capacity, int32_t* count);
/* Wait until every submitted request has finished, at most timeout_s seconds
 * (CP_ERR_TIMEOUT otherwise). */
cp_status cp_server_drain(cp_server* srv, double timeout_s);
/* Stop the server: running jobs finish, requests not yet admitted are dropped. */
cp_status cp_server_destroy(cp_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* CASCADE_H */
