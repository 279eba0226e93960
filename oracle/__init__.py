"""CPU oracle for the cascaded-prediction Krylov hot path (arXiv 2411.10143).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The product
library (``paper_2411_10143_b300``) never imports, links or executes it, and the
two share no code: this package wraps ``oracle.c`` (plain single-threaded FP64
C, built with gcc, ``-ffp-contract=off`` so every product and sum is rounded
as written) through ctypes and adds nothing but argument marshalling and a few
NumPy conveniences that follow the paper's definitions:

* ``spmv`` -- CSR SpMV by definition (Sec. I: SpMV dominates CG/GMRES time).
* ``cg`` / ``gmres`` -- Hestenes-Stiefel CG and restarted GMRES(m) with MGS and
  Givens rotations (Sec. I, Sec. IV-A).
* ``features`` -- the 15 features of Table IV (Sec. III-B-1).
* ``to_coo`` / ``to_ell`` / ``to_sell`` / ``to_hyb`` / ``to_dia`` -- canonical
  layouts of the format space (Sec. III-B-2, Sec. V-A).
* ``ir_solve`` -- FP64 iterative refinement around FP32 CG/GMRES inner solves.
* ``mlp_forward`` / ``mlp_loss_grad`` / ``adam_step`` / ``mlp_input`` -- the
  per-stage classifier (Sec. III-B-3; here a small MLP) in FP64.
* ``cascade`` -- the cascaded decision of Sec. III-C-1 (Fig. 5) from the
  stage classifiers' logits.

Parity pins for every function live in ``tests/test_oracle_*.py``.  The one
function without an independent pin (the cascade's choice of configuration is
only judged by measured SpMV time) says "parity unpinned" in its docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB = _HERE / "liboracle.so"

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_f64 = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> Path:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (no fast-math, no FP contraction)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".so.{os.getpid()}")
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = _HERE / "liboracle_omp.so"


def build_omp(force: bool = False) -> Path:
    """Compile the same ``oracle.c`` a second time with ``-fopenmp`` into
    ``liboracle_omp.so``: its SpMV rows and CG vector loops run on every host
    core.  Used only as an all-core timing baseline; parity is the serial build's."""
    if force or not _LIB_OMP.exists() or _LIB_OMP.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_OMP.with_suffix(f".so.{os.getpid()}")
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-fopenmp", "-shared", "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


_lib = None
_lib_omp = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        sig = {
            "or_spmv": (None, [_i64, _p, _p, _p, _p, _p]),
            "or_spmv_f32": (None, [_i64, _p, _p, _p, _p, _p]),
            "or_cg": (_i64, [_i64, _p, _p, _p, _p, _p, _f64, _i64, _p, _p, _i64, _p, _p]),
            "or_gmres": (_i64, [_i64, _p, _p, _p, _p, _p, _f64, _i64, _i64, _p, _i64, _p, _p]),
            "or_ir_solve": (_i64, [_i64, _p, _p, _p, _p, _p, _i32, _i64, _f64, _f64, _f64, _i64,
                                   _i64, _p, _p, _p]),
            "or_features": (None, [_i64, _i64, _p, _p, _p]),
            "or_csr_to_coo": (None, [_i64, _p, _p, _p, _p, _p, _p]),
            "or_coo_to_csr": (None, [_i64, _i64, _p, _p, _p, _p, _p, _p]),
            "or_csr_to_ell": (None, [_i64, _p, _p, _p, _i64, _i64, _p, _p]),
            "or_ell_to_csr": (None, [_i64, _i64, _i64, _p, _p, _p, _p, _p]),
            "or_sell_sizes": (_i64, [_i64, _p, _i64, _i64, _p, _p, _p]),
            "or_csr_to_sell": (None, [_i64, _p, _p, _p, _i64, _p, _p, _p, _p, _p]),
            "or_sell_to_csr": (None, [_i64, _i64, _p, _p, _p, _p, _p, _p, _p, _p]),
            "or_csr_to_hyb": (_i64, [_i64, _p, _p, _p, _i64, _i64, _p, _p, _p, _p, _p]),
            "or_hyb_to_csr": (None, [_i64, _i64, _i64, _p, _p, _i64, _p, _p, _p, _p, _p, _p]),
            "or_dia_offsets": (_i64, [_i64, _i64, _p, _p, _p]),
            "or_csr_to_dia": (None, [_i64, _p, _p, _p, _i64, _p, _p]),
            "or_mlp_nparams": (_i64, [_i64, _i64, _i64, _i64]),
            "or_mlp_forward": (None, [_i64, _i64, _i64, _i64, _i64, _p, _p, _p]),
            "or_mlp_loss_grad": (_f64, [_i64, _i64, _i64, _i64, _i64, _p, _p, _p, _p]),
            "or_mlp_loss_grad_soft": (_f64, [_i64, _i64, _i64, _i64, _i64, _p, _p, _p, _p]),
            "or_adam_step": (None, [_i64, _p, _p, _p, _p, _i64, _f64, _f64, _f64, _f64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _c(a, dtype):
    """Contiguous array of the given dtype (copy only if needed)."""
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class CSR:
    """A CSR matrix as three NumPy arrays (int32 rowptr/col, float64 val)."""

    def __init__(self, nrows, ncols, rowptr, col, val):
        self.nrows = int(nrows)
        self.ncols = int(ncols)
        self.rowptr = _c(rowptr, np.int32)
        self.col = _c(col, np.int32)
        self.val = _c(val, np.float64)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1]) if self.nrows > 0 else 0


def _as_csr(A) -> CSR:
    if isinstance(A, CSR):
        return A
    return CSR(A.nrows, A.ncols, A.rowptr, A.col, A.val)


# ---------------------------------------------------------------- SpMV / solvers
def spmv(A, x) -> np.ndarray:
    """y = A x by the CSR definition, summing each row in storage order."""
    A = _as_csr(A)
    x = _c(x, np.float64)
    y = np.empty(A.nrows, np.float64)
    lib().or_spmv(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), _ptr(x), _ptr(y))
    return y


def spmv_f32(A, x) -> np.ndarray:
    """y = A x with values, x and every partial sum rounded to FP32."""
    A = _as_csr(A)
    v32 = A.val.astype(np.float32)
    x = _c(x, np.float32)
    y = np.empty(A.nrows, np.float32)
    lib().or_spmv_f32(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(v32), _ptr(x), _ptr(y))
    return y


class SolveResult(dict):
    __getattr__ = dict.__getitem__


def cg(A, b, x0=None, tol=1e-10, maxit=100000, hist_cap=0) -> SolveResult:
    """Hestenes-Stiefel CG with a true-residual check (see ``or_cg``)."""
    A = _as_csr(A)
    b = _c(b, np.float64)
    x = np.zeros(A.nrows) if x0 is None else _c(x0, np.float64).copy()
    ah = np.zeros(max(hist_cap, 1))
    bh = np.zeros(max(hist_cap, 1))
    rel = np.zeros(1)
    st = np.zeros(1, np.int32)
    it = lib().or_cg(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), _ptr(b), _ptr(x),
                     tol, maxit, _ptr(ah), _ptr(bh), hist_cap, _ptr(rel), _ptr(st))
    k = min(it, hist_cap)
    return SolveResult(x=x, iters=int(it), relres_true=float(rel[0]), status=int(st[0]),
                       alphas=ah[:k].copy(), betas=bh[:k].copy())


def cg_all_cores(A, b, tol=1e-10, maxit=100000) -> SolveResult:
    """``cg`` run by the all-core build (``build_omp``) with x0 = 0; ``threads``
    is the OpenMP thread count it used.  A timing baseline only: its reductions
    sum in per-thread chunks, so its rounding differs from the serial oracle's."""
    global _lib_omp
    if _lib_omp is None:
        build_omp()
        L = ctypes.CDLL(str(_LIB_OMP))
        L.or_cg.restype = _i64
        L.or_cg.argtypes = [_i64, _p, _p, _p, _p, _p, _f64, _i64, _p, _p, _i64, _p, _p]
        _lib_omp = L
    A = _as_csr(A)
    b = _c(b, np.float64)
    x = np.zeros(A.nrows)
    rel = np.zeros(1)
    st = np.zeros(1, np.int32)
    it = _lib_omp.or_cg(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), _ptr(b), _ptr(x),
                        tol, maxit, None, None, 0, _ptr(rel), _ptr(st))
    threads = int(os.environ.get("OMP_NUM_THREADS", "0")) or len(os.sched_getaffinity(0))
    return SolveResult(x=x, iters=int(it), relres_true=float(rel[0]), status=int(st[0]),
                       threads=threads)


def gmres(A, b, x0=None, tol=1e-10, m=30, maxit=100000, hist_cap=0) -> SolveResult:
    """Restarted GMRES(m), MGS Arnoldi, Givens rotations (see ``or_gmres``)."""
    A = _as_csr(A)
    b = _c(b, np.float64)
    x = np.zeros(A.nrows) if x0 is None else _c(x0, np.float64).copy()
    rh = np.zeros(max(hist_cap, 1))
    rel = np.zeros(1)
    st = np.zeros(1, np.int32)
    it = lib().or_gmres(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), _ptr(b), _ptr(x),
                        tol, m, maxit, _ptr(rh), hist_cap, _ptr(rel), _ptr(st))
    k = min(it, hist_cap)
    return SolveResult(x=x, iters=int(it), relres_true=float(rel[0]), status=int(st[0]),
                       res_hist=rh[:k].copy())


def ir_solve(A, b, solver="cg", m=30, tol=1e-10, inner_tol=1e-5, max_outer=50,
             max_inner=100000, theta=0.5) -> SolveResult:
    """FP64 iterative refinement with FP32 CG/GMRES(m) inner solves (x0 = 0),
    each to relative max(inner_tol, theta tol ||b|| / ||r||)."""
    A = _as_csr(A)
    b = _c(b, np.float64)
    x = np.zeros(A.nrows)
    inner = np.zeros(1, np.int64)
    rel = np.zeros(1)
    st = np.zeros(1, np.int32)
    outer = lib().or_ir_solve(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), _ptr(b),
                              _ptr(x), 0 if solver == "cg" else 1, m, tol, inner_tol,
                              theta, max_outer, max_inner, _ptr(inner), _ptr(rel), _ptr(st))
    return SolveResult(x=x, outer=int(outer), inner_total=int(inner[0]),
                       relres_true=float(rel[0]), status=int(st[0]))


# ---------------------------------------------------------------- features
FEATURE_NAMES = ("nrows", "ncols", "nnz", "density", "mean", "sd", "cov", "max", "min",
                 "maxavg", "distavg", "clusteravg", "fill", "ndiag", "diagfill")


def features(A) -> np.ndarray:
    """The 15 features of Table IV in table order (readings in ``or_features``)."""
    A = _as_csr(A)
    f = np.zeros(15)
    lib().or_features(A.nrows, A.ncols, _ptr(A.rowptr), _ptr(A.col), _ptr(f))
    return f


# ---------------------------------------------------------------- formats
def to_coo(A):
    A = _as_csr(A)
    nnz = A.nnz
    row = np.empty(nnz, np.int32)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float64)
    lib().or_csr_to_coo(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), _ptr(row),
                        _ptr(col), _ptr(val))
    return row, col, val


def coo_to_csr(n, ncols, row, col, val) -> CSR:
    row, col, val = _c(row, np.int32), _c(col, np.int32), _c(val, np.float64)
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(len(col), np.int32)
    v = np.empty(len(col), np.float64)
    lib().or_coo_to_csr(n, len(col), _ptr(row), _ptr(col), _ptr(val), _ptr(rp), _ptr(ci), _ptr(v))
    return CSR(n, ncols, rp, ci, v)


def ell_ld(n: int) -> int:
    """Leading dimension of the ELL layouts: n rounded up to a multiple of 32."""
    return (n + 31) // 32 * 32


def to_ell(A, K=None):
    """ELL arrays (col, val), each of shape (K, ld) flattened column-major by row slot."""
    A = _as_csr(A)
    lens = np.diff(A.rowptr)
    if K is None:
        K = int(lens.max()) if A.nrows else 0
    ld = ell_ld(A.nrows)
    ecol = np.empty(K * ld, np.int32)
    eval_ = np.empty(K * ld, np.float64)
    lib().or_csr_to_ell(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), K, ld,
                        _ptr(ecol), _ptr(eval_))
    return K, ld, ecol, eval_


def ell_to_csr(n, ncols, K, ld, ecol, eval_, nnz) -> CSR:
    ecol, eval_ = _c(ecol, np.int32), _c(eval_, np.float64)
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64)
    lib().or_ell_to_csr(n, K, ld, _ptr(ecol), _ptr(eval_), _ptr(rp), _ptr(ci), _ptr(v))
    return CSR(n, ncols, rp, ci, v)


def to_sell(A, C=32, sigma=1):
    """SELL-C-sigma arrays: perm, chunk_len, chunk_ptr, col, val (see ``or_sell_sizes``)."""
    A = _as_csr(A)
    n = A.nrows
    nch = (n + C - 1) // C
    perm = np.empty(max(n, 1), np.int32)[:n]
    clen = np.empty(max(nch, 1), np.int32)[:nch]
    cptr = np.empty(nch + 1, np.int64)
    total = lib().or_sell_sizes(n, _ptr(A.rowptr), C, sigma, _ptr(perm), _ptr(clen), _ptr(cptr))
    scol = np.empty(total, np.int32)
    sval = np.empty(total, np.float64)
    lib().or_csr_to_sell(n, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), C, _ptr(perm),
                         _ptr(clen), _ptr(cptr), _ptr(scol), _ptr(sval))
    return perm, clen, cptr, scol, sval


def sell_to_csr(n, ncols, C, perm, clen, cptr, scol, sval, nnz) -> CSR:
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64)
    perm, clen = _c(perm, np.int32), _c(clen, np.int32)
    cptr, scol, sval = _c(cptr, np.int64), _c(scol, np.int32), _c(sval, np.float64)
    lib().or_sell_to_csr(n, C, _ptr(perm), _ptr(clen), _ptr(cptr), _ptr(scol), _ptr(sval),
                         _ptr(rp), _ptr(ci), _ptr(v))
    return CSR(n, ncols, rp, ci, v)


def to_hyb(A, K):
    """HYB arrays: ELL part (width K) and COO remainder (row, col, val)."""
    A = _as_csr(A)
    ld = ell_ld(A.nrows)
    nc = lib().or_csr_to_hyb(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), K, ld,
                             None, None, None, None, None)
    ecol = np.empty(K * ld, np.int32)
    eval_ = np.empty(K * ld, np.float64)
    crow = np.empty(nc, np.int32)
    ccol = np.empty(nc, np.int32)
    cval = np.empty(nc, np.float64)
    lib().or_csr_to_hyb(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), K, ld, _ptr(ecol),
                        _ptr(eval_), _ptr(crow), _ptr(ccol), _ptr(cval))
    return ld, ecol, eval_, crow, ccol, cval


def hyb_to_csr(n, ncols, K, ld, ecol, eval_, crow, ccol, cval, nnz) -> CSR:
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64)
    args = [_c(ecol, np.int32), _c(eval_, np.float64), _c(crow, np.int32),
            _c(ccol, np.int32), _c(cval, np.float64)]
    lib().or_hyb_to_csr(n, K, ld, _ptr(args[0]), _ptr(args[1]), len(args[2]), _ptr(args[2]),
                        _ptr(args[3]), _ptr(args[4]), _ptr(rp), _ptr(ci), _ptr(v))
    return CSR(n, ncols, rp, ci, v)


def to_dia(A):
    """DIA arrays: ascending offsets (col - row) and values [ndiag][nrows] (0.0 where absent)."""
    A = _as_csr(A)
    offs = np.empty(max(A.nrows + A.ncols - 1, 1), np.int32)
    nd = lib().or_dia_offsets(A.nrows, A.ncols, _ptr(A.rowptr), _ptr(A.col), _ptr(offs))
    offs = offs[:nd].copy()
    data = np.empty(nd * A.nrows, np.float64)
    lib().or_csr_to_dia(A.nrows, _ptr(A.rowptr), _ptr(A.col), _ptr(A.val), nd, _ptr(offs),
                        _ptr(data))
    return offs, data


# ---------------------------------------------------------------- predictor MLP
def mlp_nparams(d, h1, h2, k) -> int:
    return int(lib().or_mlp_nparams(d, h1, h2, k))


def mlp_forward(P, X, dims) -> np.ndarray:
    """Logits of the MLP d -> h1 -> h2 -> k (ReLU hidden layers), FP64."""
    d, h1, h2, k = dims
    P = _c(P, np.float64)
    X = _c(X, np.float64).reshape(-1, d)
    out = np.empty((X.shape[0], k))
    lib().or_mlp_forward(X.shape[0], d, h1, h2, k, _ptr(P), _ptr(X), _ptr(out))
    return out


def mlp_loss_grad(P, X, labels, dims):
    """(mean softmax cross-entropy, gradient in P's flat layout), FP64."""
    d, h1, h2, k = dims
    P = _c(P, np.float64)
    X = _c(X, np.float64).reshape(-1, d)
    lab = _c(labels, np.int32)
    dP = np.empty_like(P)
    loss = lib().or_mlp_loss_grad(X.shape[0], d, h1, h2, k, _ptr(P), _ptr(X), _ptr(lab), _ptr(dP))
    return float(loss), dP


def mlp_loss_grad_soft(P, X, targets, dims):
    """(mean cross-entropy against target distributions, gradient), FP64."""
    d, h1, h2, k = dims
    P = _c(P, np.float64)
    X = _c(X, np.float64).reshape(-1, d)
    Q = _c(targets, np.float64).reshape(X.shape[0], k)
    dP = np.empty_like(P)
    loss = lib().or_mlp_loss_grad_soft(X.shape[0], d, h1, h2, k, _ptr(P), _ptr(X), _ptr(Q),
                                       _ptr(dP))
    return float(loss), dP


def adam_step(P, G, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays P, m, v."""
    for a in (P, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    G = _c(G, np.float64)
    lib().or_adam_step(len(P), _ptr(P), _ptr(G), _ptr(m), _ptr(v), t, lr, b1, b2, eps)


def mlp_input(f, mu, sd) -> np.ndarray:
    """Classifier input from the 15 features: z_j = (log(1 + f_j) - mu_j) / sd_j, FP64.

    All 15 Table IV features are non-negative; the log compresses their ranges
    (nnz spans 1e3..1e8) before standardisation with the training set's
    per-feature mean ``mu`` and standard deviation ``sd``.
    """
    f = np.asarray(f, np.float64)
    return (np.log1p(f) - np.asarray(mu, np.float64)) / np.asarray(sd, np.float64)


# ---------------------------------------------------------------- cascade
FORMATS = ("CSR", "COO", "ELL", "SELL", "HYB", "DIA")


def cascade(format_logits, algo_logits=None, tpv_logits=None, sell_logits=None):
    """The cascaded decision of Sec. III-C-1 (Fig. 5) from per-stage logits.

    Stage 1 picks the format (argmax over FORMATS).  Only if it is CSR does
    stage 2 pick the CSR algorithm (scalar, vector, merge); only if that is the
    vector kernel does stage 3 pick threads per row (2, 4, 8, 16, 32).  If the
    format is SELL, stage 2's place is taken by the sigma classifier.
    Returns (format, algo, param) indices, -1 where a stage does not apply.

    Parity unpinned: which configuration is *right* is judged by measured
    SpMV time, not by a closed form; this function only fixes the control flow.
    """
    fmt = int(np.argmax(format_logits))
    algo, param = -1, -1
    if FORMATS[fmt] == "CSR" and algo_logits is not None:
        algo = int(np.argmax(algo_logits))
        if algo == 1 and tpv_logits is not None:
            param = int(np.argmax(tpv_logits))
    elif FORMATS[fmt] == "SELL" and sell_logits is not None:
        param = int(np.argmax(sell_logits))
    return fmt, algo, param
