"""Python binding of libcascade (include/cascade.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts
NumPy arrays and torch tensors into pointers and sizes, calls the C ABI and
turns a non-zero cp_status into a :class:`CascadeError`.  PyTorch supplies
device memory and streams.  There is no CPU fallback: if ``libcascade.so`` is
missing or no GPU is present the calls raise.

Names follow the C ABI without the ``cp_`` prefix: :class:`Context`
(cp_create / cp_destroy), :meth:`Context.csr_load`, :meth:`Matrix.spmv`,
:meth:`Matrix.features`, :meth:`Matrix.convert`, :meth:`Matrix.predict`,
:meth:`Matrix.solve_cg`, :meth:`Matrix.solve_gmres`, ...
"""
from __future__ import annotations

import ctypes
from ctypes import POINTER, Structure, byref, c_char_p, c_double, c_float, c_int32, c_int64
from ctypes import c_uint64, c_void_p
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "libcascade.so"

OK, ERR_INVALID, ERR_OOM, ERR_FOOTPRINT, ERR_NOT_CONVERGED, ERR_BREAKDOWN = range(6)
ERR_TIMEOUT, ERR_CUDA, ERR_CANCELLED, ERR_UNSUPPORTED = range(6, 10)
FMT_CSR, FMT_COO, FMT_ELL, FMT_SELL, FMT_HYB, FMT_DIA = range(6)
FORMATS = ("CSR", "COO", "ELL", "SELL", "HYB", "DIA")
ALGO_SCALAR, ALGO_VECTOR, ALGO_MERGE = range(3)
MODE_PLAIN, MODE_SEQUENTIAL, MODE_ASYNC = range(3)
PREC_FP64, PREC_FP32_IR = range(2)
DTYPE_F64, DTYPE_F32 = range(2)
STAGE_FORMAT, STAGE_CSR_ALGO, STAGE_CSR_TPV, STAGE_SELL_SIGMA, STAGE_BATCH_TPR = range(5)
STAGE_CLASSES = (6, 3, 5, 4, 3)
BATCH_TPR_CLASSES = (1, 4, 16)  # threads per row of the batched solve, by class
TPV_CLASSES = (2, 4, 8, 16, 32)
SIGMA_CLASSES = (1, 32, 1024, 8192)
ARR = dict(COO_ROW=0, ELL_COL=1, ELL_VAL=2, SELL_PERM=3, SELL_CHUNK_LEN=4, SELL_CHUNK_PTR=5,
           SELL_COL=6, SELL_VAL=7, HYB_ELL_COL=8, HYB_ELL_VAL=9, HYB_COO_ROW=10,
           HYB_COO_COL=11, HYB_COO_VAL=12, DIA_OFFSETS=13, DIA_VAL=14)


class CascadeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cascade error {status}: {msg}")
        self.status = status


class Config(Structure):
    _fields_ = [("fmt", c_int32), ("algo", c_int32), ("tpv", c_int32), ("sell_c", c_int32),
                ("sell_sigma", c_int32), ("hyb_k", c_int32)]

    def as_tuple(self):
        return (self.fmt, self.algo, self.tpv, self.sell_c, self.sell_sigma, self.hyb_k)

    def __repr__(self):
        name = FORMATS[self.fmt]
        if self.fmt == FMT_CSR:
            name += ("-scalar", f"-vector{self.tpv}", "-merge")[self.algo]
        elif self.fmt == FMT_SELL:
            name += f"-{self.sell_c}-{self.sell_sigma}"
        elif self.fmt == FMT_HYB:
            name += f"-K{self.hyb_k}"
        return name


def config(fmt="CSR", algo=ALGO_SCALAR, tpv=8, sigma=1, hyb_k=0) -> Config:
    """A cp_config; fmt by name or index."""
    f = FORMATS.index(fmt) if isinstance(fmt, str) else int(fmt)
    return Config(f, algo, tpv, 32, sigma, hyb_k)


class SolveOpts(Structure):
    _fields_ = [("tol", c_double), ("maxit", c_int32), ("restart", c_int32), ("mode", c_int32),
                ("precision", c_int32), ("inner_tol", c_double), ("max_outer", c_int32),
                ("check_every", c_int32), ("profile", c_int32), ("iteration_kernel", c_int32),
                ("force", POINTER(Config)), ("wait_limit_ms", c_double),
                ("persist_chunk", c_int32), ("gmres_orth", c_int32), ("ir_theta", c_double)]


class SolveInfo(Structure):
    _fields_ = [("iters", c_int32), ("outer_iters", c_int32), ("switch_iter", c_int32 * 3),
                ("n_spmv", c_int32), ("n_launches", c_int32), ("status", c_int32),
                ("relres_true", c_double), ("final_cfg", Config), ("t_features_ms", c_float),
                ("t_predict_ms", c_float * 3), ("t_convert_ms", c_float),
                ("t_total_ms", c_float), ("t_spmv_ms", c_float), ("t_persist_ms", c_float),
                ("persist_iters", c_int32), ("t_persist_last_ms", c_float),
                ("persist_last_iters", c_int32), ("gate_declined", c_int32),
                ("gate_remaining", c_float), ("gate_cost_spmvs", c_float),
                ("side_status", c_int32), ("persist_launches", c_int32)]

    def as_dict(self):
        return dict(iters=self.iters, outer_iters=self.outer_iters,
                    switch_iter=list(self.switch_iter), n_spmv=self.n_spmv,
                    n_launches=self.n_launches, status=self.status,
                    relres_true=self.relres_true, final_cfg=repr(self.final_cfg),
                    t_features_ms=self.t_features_ms, t_predict_ms=list(self.t_predict_ms),
                    t_convert_ms=self.t_convert_ms, t_total_ms=self.t_total_ms,
                    t_spmv_ms=self.t_spmv_ms, t_persist_ms=self.t_persist_ms,
                    persist_iters=self.persist_iters, t_persist_last_ms=self.t_persist_last_ms,
                    persist_last_iters=self.persist_last_iters,
                    gate_declined=self.gate_declined, gate_remaining=self.gate_remaining,
                    gate_cost_spmvs=self.gate_cost_spmvs, side_status=self.side_status,
                    persist_launches=self.persist_launches)


class Gate(Structure):
    """cp_gate: the cost-aware switching figures (arrays indexed by FORMATS)."""
    _fields_ = [("speedup", c_double * 6), ("conv_a_ms", c_double * 6),
                ("conv_b_ms", c_double * 6), ("spmv_a_ms", c_double), ("spmv_b_ms", c_double),
                ("feat_a_ms", c_double), ("feat_b_ms", c_double), ("small_rows", c_int64),
                ("enabled", c_int32)]

    @classmethod
    def from_dict(cls, d, enabled=True):
        g = cls()
        for i in range(6):
            g.speedup[i] = float(d["speedup"][i])
            g.conv_a_ms[i] = float(d["conv_a_ms"][i])
            g.conv_b_ms[i] = float(d["conv_b_ms"][i])
        g.spmv_a_ms = float(d["spmv_a_ms"])
        g.spmv_b_ms = float(d["spmv_b_ms"])
        g.feat_a_ms = float(d.get("feat_a_ms", 0.0))
        g.feat_b_ms = float(d.get("feat_b_ms", 0.0))
        g.small_rows = int(d.get("small_rows", 100_000))
        g.enabled = 1 if enabled else 0
        return g


def gate_decide(gate: Gate, fmt, nnz, iters, res0, res, target):
    """cp_gate_decide (host only): (switch?, remaining iterations, cost in SpMVs)."""
    rem, cost = c_double(0.0), c_double(0.0)
    go = lib().cp_gate_decide(byref(gate), int(fmt), int(nnz), int(iters), float(res0),
                              float(res), float(target), byref(rem), byref(cost))
    return bool(go), rem.value, cost.value


def gate_payback(gate: Gate, fmt, nnz):
    """cp_gate_payback (host only): default-kernel iterations to pay back the
    conversion to ``fmt``."""
    return lib().cp_gate_payback(byref(gate), int(fmt), int(nnz))


def _neighbours(z, speedup, mu, sd):
    z = _np(z, np.float32).reshape(-1, 15)
    speedup = _np(speedup, np.float32).reshape(-1, 6)
    if len(z) != len(speedup):
        raise ValueError("z and speedup must have one row per training matrix")
    return z, speedup, _np(mu, np.float64).reshape(15), _np(sd, np.float64).reshape(15)


def gate_knn_speedup(z, speedup, mu, sd, features, fmt, k=7) -> float:
    """cp_gate_knn_speedup (host only): format fmt's median speedup over the k
    training matrices nearest to `features` (15 Table IV features)."""
    z, speedup, mu, sd = _neighbours(z, speedup, mu, sd)
    f = _np(features, np.float64).reshape(15)
    out = c_double(0.0)
    _check(lib().cp_gate_knn_speedup(len(z), int(k), _ptr(mu), _ptr(sd), _ptr(z), _ptr(speedup),
                                     _ptr(f), int(fmt), byref(out)))
    return out.value


class ServerOpts(Structure):
    _fields_ = [("tol", c_double), ("inner_tol", c_double), ("restart", c_int32),
                ("maxit", c_int32), ("small_max_n", c_int32), ("max_batch", c_int32),
                ("lanes", c_int32), ("mode", c_int32), ("mem_budget", c_int64),
                ("small_max_n_gmres", c_int32), ("ir_theta", c_double)]


class Request(Structure):
    _fields_ = [("id", c_int64), ("mat", c_void_p), ("solver", c_int32), ("reserved", c_int32),
                ("b", c_void_p), ("x", c_void_p)]


class Result(Structure):
    _fields_ = [("id", c_int64), ("status", c_int32), ("iters", c_int32), ("batched", c_int32),
                ("lane", c_int32), ("relres_true", c_double), ("t_submit_ms", c_double),
                ("t_start_ms", c_double), ("t_done_ms", c_double)]


_p = c_void_p
# the ctypes mirrors of the header's structs, in cp_abi_sizeof's order
ABI_STRUCTS = (Config, SolveOpts, SolveInfo, Gate, ServerOpts, Request, Result)

_SIGS = {
    "cp_config_default": (None, [POINTER(Config)]),
    "cp_solve_opts_default": (None, [POINTER(SolveOpts)]),
    "cp_last_error": (c_char_p, []),
    "cp_abi_sizeof": (c_int64, [c_int32]),
    "cp_create": (c_int32, [POINTER(_p), c_int32, _p, _p]),
    "cp_destroy": (c_int32, [_p]),
    "cp_ctx_launch_count": (c_int32, [_p, POINTER(c_int64)]),
    "cp_set_format_budget": (c_int32, [_p, c_int64]),
    "cp_csr_load": (c_int32, [_p, c_int64, c_int64, c_int64, _p, _p, _p, c_int32, POINTER(_p)]),
    "cp_mat_free": (c_int32, [_p]),
    "cp_mat_reset": (c_int32, [_p]),
    "cp_features": (c_int32, [_p, _p, _p]),
    "cp_convert": (c_int32, [_p, _p, POINTER(Config)]),
    "cp_format_dims": (c_int32, [_p, _p, POINTER(Config), _p]),
    "cp_format_export": (c_int32, [_p, _p, POINTER(Config), c_int32, _p, c_int64,
                                   POINTER(c_int64)]),
    "cp_spmv": (c_int32, [_p, _p, POINTER(Config), c_int32, c_double, _p, c_double, _p]),
    "cp_spmv_csr_merge_noalloc": (c_int32, [c_int64, c_int64, c_int64, _p, _p, _p, _p, _p, _p]),
    "cp_mlp_nparams": (c_int64, [c_int32, c_int32, c_int32, c_int32]),
    "cp_mlp_scratch_floats": (c_int64, [c_int64, c_int32, c_int32, c_int32, c_int32]),
    "cp_mlp_forward": (c_int32, [_p, c_int64, c_int32, c_int32, c_int32, c_int32, _p, _p, _p, _p]),
    "cp_mlp_loss_grad": (c_int32, [_p, c_int64, c_int32, c_int32, c_int32, c_int32, _p, _p, _p,
                                   _p, _p, _p]),
    "cp_mlp_loss_grad_soft": (c_int32, [_p, c_int64, c_int32, c_int32, c_int32, c_int32, _p, _p,
                                        _p, _p, _p, _p]),
    "cp_model_train_soft": (c_int32, [_p, c_int32, c_int64, _p, _p, c_int32, c_int32, c_int32,
                                      c_int32, c_float, c_uint64, POINTER(c_float)]),
    "cp_adam_step": (c_int32, [_p, c_int64, _p, _p, _p, _p, c_int32, c_float, c_float, c_float,
                               c_float]),
    "cp_model_load": (c_int32, [_p, c_int32, c_int32, c_int32, c_int32, _p, _p, _p]),
    "cp_model_get": (c_int32, [_p, c_int32, _p, _p, c_int64, _p, _p]),
    "cp_model_train": (c_int32, [_p, c_int32, c_int64, _p, _p, c_int32, c_int32, c_int32,
                                 c_int32, c_float, c_uint64, POINTER(c_float)]),
    "cp_predict": (c_int32, [_p, _p, POINTER(Config), _p]),
    "cp_predict_stage": (c_int32, [_p, c_int32, _p, _p, POINTER(c_int32)]),
    "cp_solve_cg": (c_int32, [_p, _p, _p, _p, POINTER(SolveOpts), POINTER(SolveInfo)]),
    "cp_solve_gmres": (c_int32, [_p, _p, _p, _p, POINTER(SolveOpts), POINTER(SolveInfo)]),
    "cp_batch_solve": (c_int32, [_p, c_int32, _p, _p, _p, _p, POINTER(SolveOpts), c_int32,
                                 c_int32, _p]),
    "cp_gate_set": (c_int32, [_p, _p]),
    "cp_inject_side_failure": (c_int32, [_p, c_int32]),
    "cp_warmup": (c_int32, [_p]),
    "cp_fp64_fma_rate": (c_int32, [_p, POINTER(c_double)]),
    "cp_gate_decide": (c_int32, [_p, c_int32, c_int64, c_int32, c_double, c_double, c_double,
                                 POINTER(c_double), POINTER(c_double)]),
    "cp_gate_payback": (c_double, [_p, c_int32, c_int64]),
    "cp_gate_knn_speedup": (c_int32, [c_int32, c_int32, _p, _p, _p, _p, _p, c_int32,
                                      POINTER(c_double)]),
    "cp_gate_set_neighbours": (c_int32, [_p, c_int32, c_int32, _p, _p, _p, _p]),
    "cp_batch_tune": (c_int32, [_p, c_int32, _p, _p, _p, POINTER(SolveOpts), POINTER(c_int32),
                                POINTER(c_int32), POINTER(c_int32), _p, POINTER(c_float)]),
    "cp_batch_schedule": (c_int32, [_p, c_int64, c_int32, POINTER(c_int32), POINTER(c_int32),
                                    POINTER(c_int32)]),
    "cp_batch_tpr": (c_int32, [_p, _p, POINTER(c_int32)]),
    "cp_server_opts_default": (None, [POINTER(ServerOpts)]),
    "cp_server_create": (c_int32, [_p, POINTER(ServerOpts), POINTER(_p)]),
    "cp_server_submit": (c_int32, [_p, POINTER(Request)]),
    "cp_server_poll": (c_int32, [_p, _p, c_int32, POINTER(c_int32)]),
    "cp_server_drain": (c_int32, [_p, c_double]),
    "cp_server_destroy": (c_int32, [_p]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Load libcascade.so (built in-tree by ``paper_2411_10143_b300.build``)."""
    global _lib
    if _lib is None:
        if not _LIB_PATH.exists():
            raise CascadeError(ERR_CUDA, f"{_LIB_PATH.name} is not built; run build.build()")
        L = ctypes.CDLL(str(_LIB_PATH))
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        for which, cls in enumerate(ABI_STRUCTS):
            want = L.cp_abi_sizeof(which)
            if want != ctypes.sizeof(cls):
                raise CascadeError(ERR_INVALID, f"{cls.__name__} is {ctypes.sizeof(cls)} bytes, "
                                                f"the library's struct {want}: rebuild or fix "
                                                "the binding")
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        msg = lib().cp_last_error()
        raise CascadeError(status, msg.decode() if msg else "")


def _ptr(a):
    """Address of a torch tensor or NumPy array (must stay alive during the call)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return c_void_p(a.data_ptr())
    return a.ctypes.data_as(c_void_p)


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def spmv_csr_merge_noalloc(nrows, ncols, rowptr, col, val, x, y, stream=None, nnz=None):
    """cp_spmv_csr_merge_noalloc on torch CUDA tensors: y = A x with no device
    allocation (fixed library scratch; see cascade.h for its limit and for why
    overlapping calls must be serialised).

    The C entry point does not validate the CSR, so the arrays' types, device,
    layout and lengths are checked here before any pointer reaches a kernel:
    int32 rowptr / col, float64 val / x / y, contiguous, on the current CUDA
    device, rowptr of nrows + 1 entries, col and val of at least nnz entries,
    x of at least ncols and y of at least nrows.  ``nnz`` defaults to
    ``col.numel()``; pass it when col / val are slices of a larger arena buffer.
    """
    import torch
    nrows, ncols = int(nrows), int(ncols)
    nnz = int(col.numel()) if nnz is None else int(nnz)
    dev = torch.cuda.current_device()
    for name, t, dt in (("rowptr", rowptr, torch.int32), ("col", col, torch.int32),
                        ("val", val, torch.float64), ("x", x, torch.float64),
                        ("y", y, torch.float64)):
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_cuda or \
                t.device.index != dev or not t.is_contiguous():
            raise CascadeError(ERR_INVALID, f"spmv_csr_merge_noalloc: {name} must be a "
                               f"contiguous {dt} tensor on cuda:{dev}")
    if nrows < 1 or ncols < 1 or nnz < 0:
        raise CascadeError(ERR_INVALID, "spmv_csr_merge_noalloc: sizes out of range")
    if rowptr.numel() != nrows + 1 or col.numel() < nnz or val.numel() < nnz or \
            x.numel() < ncols or y.numel() < nrows:
        raise CascadeError(ERR_INVALID, "spmv_csr_merge_noalloc: an array is shorter than "
                           "its size argument (rowptr nrows+1, col/val nnz, x ncols, y nrows)")
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().cp_spmv_csr_merge_noalloc(nrows, ncols, nnz, _ptr(rowptr), _ptr(col), _ptr(val),
                                           _ptr(x), _ptr(y), c_void_p(s) if s else None))


def default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().cp_solve_opts_default(byref(o))
    for k, v in kw.items():
        if k == "force":
            continue
        _set_field(o, k, v)
    return o


def _set_field(o, k, v):
    """Sets a field of a ctypes struct; an unknown name is an error rather than
    a new Python attribute the library would never see."""
    if k not in {f[0] for f in type(o)._fields_}:
        raise TypeError(f"{type(o).__name__} has no field {k!r}")
    setattr(o, k, v)


class _Ordered:
    """Orders the library's main stream after torch's current stream on entry and
    torch's current stream after the library's main stream on exit (event waits),
    so tensors filled before a call are complete when the library reads them and
    the library's results are complete before later torch work reads them."""

    def __init__(self, ctx):
        self.ctx = ctx

    def __enter__(self):
        import torch
        cur = torch.cuda.current_stream(self.ctx.device)
        if cur != self.ctx.stream:
            self.ctx.stream.wait_stream(cur)
        return self

    def __exit__(self, *exc):
        import torch
        cur = torch.cuda.current_stream(self.ctx.device)
        if cur != self.ctx.stream:
            cur.wait_stream(self.ctx.stream)
        return False


class Context:
    """cp_create / cp_destroy.  ``main_stream`` / ``side_stream`` are torch CUDA
    streams (or None)."""

    def __init__(self, device: int = 0, main_stream=None, side_stream=None):
        """Without ``main_stream`` the library gets a torch stream of its own (never
        the legacy default stream, which serialises with other streams' allocations
        and copies) and every call is ordered against torch's current stream by
        event waits.  The side stream defaults to a library-owned non-blocking
        stream."""
        import torch
        self._h = c_void_p()
        self.device = device
        if main_stream is None or main_stream.cuda_stream == 0:
            main_stream = torch.cuda.Stream(device)
        self.stream = main_stream
        self._streams = (main_stream, side_stream)  # keep them alive
        ms = c_void_p(main_stream.cuda_stream)
        ss = c_void_p(side_stream.cuda_stream) if side_stream is not None else None
        _check(lib().cp_create(byref(self._h), device, ms, ss))

    def ordered(self):
        return _Ordered(self)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _check(lib().cp_destroy(self._h))
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        c = c_int64()
        _check(lib().cp_ctx_launch_count(self._h, byref(c)))
        return c.value

    def set_format_budget(self, nbytes: int):
        _check(lib().cp_set_format_budget(self._h, int(nbytes)))

    def csr_load(self, nrows, ncols, rowptr, col, val) -> "Matrix":
        """Copy a CSR matrix (NumPy host arrays or torch CUDA tensors) into the library."""
        on_dev = hasattr(rowptr, "is_cuda") and rowptr.is_cuda
        if not on_dev:
            rowptr, col, val = _np(rowptr, np.int32), _np(col, np.int32), _np(val, np.float64)
        nnz = int(col.numel() if on_dev else col.size)
        h = c_void_p()
        with self.ordered():
            _check(lib().cp_csr_load(self._h, int(nrows), int(ncols), nnz, _ptr(rowptr),
                                     _ptr(col), _ptr(val), 1 if on_dev else 0, byref(h)))
        return Matrix(self, h, int(nrows), int(ncols), nnz)

    def load(self, A) -> "Matrix":
        """csr_load of a matrix object with nrows, ncols, rowptr, col, val."""
        return self.csr_load(A.nrows, A.ncols, A.rowptr, A.col, A.val)

    # ---------------------------------------------------------------- predictors
    def model_load(self, stage, h1, h2, k, params, mu, sd):
        params, mu, sd = _np(params, np.float32), _np(mu, np.float32), _np(sd, np.float32)
        _check(lib().cp_model_load(self._h, stage, h1, h2, k, _ptr(params), _ptr(mu), _ptr(sd)))

    def model_get(self, stage):
        dims = np.zeros(4, np.int32)
        _check(lib().cp_model_get(self._h, stage, _ptr(dims), None, 0, None, None))
        n = int(lib().cp_mlp_nparams(*[int(v) for v in dims]))
        params = np.zeros(n, np.float32)
        mu = np.zeros(15, np.float32)
        sd = np.zeros(15, np.float32)
        _check(lib().cp_model_get(self._h, stage, _ptr(dims), _ptr(params), n, _ptr(mu), _ptr(sd)))
        return dict(dims=dims.tolist(), params=params, mu=mu, sd=sd)

    def predict_stage(self, stage, features):
        """cp_predict_stage: (logits, pick) of one installed cascade stage on a
        15-feature host vector."""
        f = _np(features, np.float64).reshape(15)
        logits = np.zeros(STAGE_CLASSES[stage], np.float32)
        pick = c_int32()
        _check(lib().cp_predict_stage(self._h, stage, _ptr(f), _ptr(logits), byref(pick)))
        return logits, pick.value

    def model_train(self, stage, F, labels, h1=32, h2=32, epochs=2000, lr=3e-3, seed=1):
        F = _np(F, np.float64).reshape(-1, 15)
        lab = _np(labels, np.int32)
        loss = c_float()
        _check(lib().cp_model_train(self._h, stage, F.shape[0], _ptr(F), _ptr(lab), h1, h2,
                                    STAGE_CLASSES[stage], epochs, lr, seed, byref(loss)))
        return loss.value

    def model_train_soft(self, stage, F, targets, h1=32, h2=32, epochs=2000, lr=3e-3, seed=1):
        """cp_model_train_soft: train a stage on target distributions targets[N][k]."""
        F = _np(F, np.float64).reshape(-1, 15)
        Q = _np(targets, np.float32).reshape(F.shape[0], STAGE_CLASSES[stage])
        loss = c_float()
        _check(lib().cp_model_train_soft(self._h, stage, F.shape[0], _ptr(F), _ptr(Q), h1, h2,
                                         STAGE_CLASSES[stage], epochs, lr, seed, byref(loss)))
        return loss.value

    def mlp_forward(self, dims, params, X, logits, scratch):
        d, h1, h2, k = dims
        with self.ordered():
            _check(lib().cp_mlp_forward(self._h, X.shape[0], d, h1, h2, k, _ptr(params),
                                        _ptr(X), _ptr(logits), _ptr(scratch)))

    def mlp_loss_grad(self, dims, params, X, labels, loss, grad, scratch):
        d, h1, h2, k = dims
        with self.ordered():
            _check(lib().cp_mlp_loss_grad(self._h, X.shape[0], d, h1, h2, k, _ptr(params),
                                          _ptr(X), _ptr(labels), _ptr(loss), _ptr(grad),
                                          _ptr(scratch)))

    def mlp_loss_grad_soft(self, dims, params, X, targets, loss, grad, scratch):
        d, h1, h2, k = dims
        with self.ordered():
            _check(lib().cp_mlp_loss_grad_soft(self._h, X.shape[0], d, h1, h2, k, _ptr(params),
                                               _ptr(X), _ptr(targets), _ptr(loss), _ptr(grad),
                                               _ptr(scratch)))

    def adam_step(self, params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        with self.ordered():
            _check(lib().cp_adam_step(self._h, params.numel(), _ptr(params), _ptr(grad), _ptr(m),
                                      _ptr(v), t, lr, b1, b2, eps))

    def batch_solve(self, mats, solvers, bs, xs, opts=None, threads=0, threads_per_row=0,
                    raise_on_error=True):
        """cp_batch_solve: many small systems in one persistent launch.  mats:
        Matrix list; solvers: 0 (CG) / 1 (GMRES) per system; bs, xs: torch CUDA
        float64 tensors (xs: x0 in, solutions out); threads / threads_per_row: the
        launch shape (0: the class's schedule).  Returns the SolveInfo list."""
        n = len(mats)
        hm = (c_void_p * n)(*[m._h.value for m in mats])
        hs = np.ascontiguousarray(solvers, np.int32)
        hb = (c_void_p * n)(*[t.data_ptr() for t in bs])
        hx = (c_void_p * n)(*[t.data_ptr() for t in xs])
        infos = (SolveInfo * n)()
        o = opts if opts is not None else default_opts(precision=PREC_FP32_IR)
        with self.ordered():
            st = lib().cp_batch_solve(self._h, n, hm, _ptr(hs), hb, hx, byref(o), threads,
                                      threads_per_row, infos)
        if raise_on_error:
            _check(st)
        return list(infos)

    BATCH_THREADS = (128, 256, 512, 1024)
    BATCH_TPV = (1, 4, 16)

    def batch_tune(self, mats, solvers, bs, opts=None, with_order=False):
        """cp_batch_tune: time every launch shape (128/256/512/1024 threads per
        system x 1/4/16 threads per row) on this batch (scratch solutions), then
        the best shape in the caller's order, and record the fastest for its
        class.  Returns ((threads, threads per row), {(threads, threads per row):
        ms}); with_order adds (packing order, ms of the best shape in the
        caller's order)."""
        n = len(mats)
        hm = (c_void_p * n)(*[m._h.value for m in mats])
        hs = np.ascontiguousarray(solvers, np.int32)
        hb = (c_void_p * n)(*[t.data_ptr() for t in bs])
        best, best_tpv, best_order = c_int32(0), c_int32(0), c_int32(0)
        ms = np.zeros(12, np.float32)
        ms_order = c_float(0.0)
        o = opts if opts is not None else default_opts(precision=PREC_FP32_IR)
        with self.ordered():
            _check(lib().cp_batch_tune(self._h, n, hm, _ptr(hs), hb, byref(o), byref(best),
                                       byref(best_tpv), byref(best_order), _ptr(ms),
                                       byref(ms_order)))
        times = {(t, r): float(ms[3 * i + j]) for i, t in enumerate(self.BATCH_THREADS)
                 for j, r in enumerate(self.BATCH_TPV)}
        if with_order:
            return (best.value, best_tpv.value), times, (best_order.value, ms_order.value)
        return (best.value, best_tpv.value), times

    def fp64_fma_rate(self):
        """cp_fp64_fma_rate: measured FP64 FMAs per second of this GPU."""
        r = c_double()
        with self.ordered():
            _check(lib().cp_fp64_fma_rate(self._h, byref(r)))
        return r.value

    def warmup(self):
        """cp_warmup: launch every solve-path kernel once on a small system, so that
        no timed solve pays a kernel's one-time first-launch cost."""
        with self.ordered():
            _check(lib().cp_warmup(self._h))

    def inject_side_failure(self, point):
        """cp_inject_side_failure (tests): the next solve's side thread fails at point."""
        _check(lib().cp_inject_side_failure(self._h, int(point)))

    def gate_set(self, gate: "Gate"):
        """cp_gate_set: install (gate.enabled = 1) or disable the cost-aware switch."""
        _check(lib().cp_gate_set(self._h, byref(gate)))

    def gate_set_neighbours(self, z=None, speedup=None, mu=None, sd=None, k=7):
        """cp_gate_set_neighbours: per-matrix speedups for the gate (None removes them)."""
        if z is None:
            _check(lib().cp_gate_set_neighbours(self._h, 0, 0, None, None, None, None))
            return
        z, speedup, mu, sd = _neighbours(z, speedup, mu, sd)
        _check(lib().cp_gate_set_neighbours(self._h, len(z), int(k), _ptr(mu), _ptr(sd), _ptr(z),
                                            _ptr(speedup)))

    def batch_tpr(self, mat):
        """cp_batch_tpr: the threads per row the BATCH_TPR classifier gives the
        systems of ``mat`` in a batched solve (0 without a model)."""
        t = c_int32(0)
        with self.ordered():
            _check(lib().cp_batch_tpr(self._h, mat._h, byref(t)))
        return t.value

    def batch_schedule(self, mean_rows, has_gmres=False, with_order=False):
        """(threads per system, threads per row) cp_batch_solve(threads=0) uses for
        a batch class; with_order adds the packing order (0: largest first, 1:
        the caller's order)."""
        t, r, o = c_int32(0), c_int32(0), c_int32(0)
        _check(lib().cp_batch_schedule(self._h, int(mean_rows), 1 if has_gmres else 0, byref(t),
                                       byref(r), byref(o)))
        return (t.value, r.value, o.value) if with_order else (t.value, r.value)

    @staticmethod
    def mlp_nparams(d, h1, h2, k):
        return int(lib().cp_mlp_nparams(d, h1, h2, k))

    @staticmethod
    def mlp_scratch_floats(N, d, h1, h2, k):
        return int(lib().cp_mlp_scratch_floats(N, d, h1, h2, k))


class Matrix:
    """A cp_mat: library-owned device copy of a CSR matrix and its converted formats."""

    def __init__(self, ctx: Context, h, nrows, ncols, nnz):
        self.ctx, self._h = ctx, h
        self.nrows, self.ncols, self.nnz = nrows, ncols, nnz

    def free(self):
        if self._h:
            _check(lib().cp_mat_free(self._h))
            self._h = c_void_p()

    def __del__(self):
        try:
            if self.ctx._h:
                self.free()
        except Exception:
            pass

    def reset(self):
        """Drop converted formats and cached features (cp_mat_reset)."""
        _check(lib().cp_mat_reset(self._h))

    def features(self) -> np.ndarray:
        out = np.zeros(15)
        _check(lib().cp_features(self.ctx.handle, self._h, _ptr(out)))
        return out

    def convert(self, cfg: Config):
        _check(lib().cp_convert(self.ctx.handle, self._h, byref(cfg)))

    def format_dims(self, cfg: Config):
        d = np.zeros(4, np.int64)
        _check(lib().cp_format_dims(self.ctx.handle, self._h, byref(cfg), _ptr(d)))
        return d.tolist()

    def format_export(self, cfg: Config, array: str, dtype) -> np.ndarray:
        nb = c_int64()
        probe = np.zeros(1, np.uint8)
        st = lib().cp_format_export(self.ctx.handle, self._h, byref(cfg), ARR[array], _ptr(probe),
                                    0, byref(nb))
        if st not in (OK, ERR_INVALID):
            _check(st)
        out = np.zeros(max(nb.value, 1), np.uint8)
        _check(lib().cp_format_export(self.ctx.handle, self._h, byref(cfg), ARR[array], _ptr(out),
                                      out.size, byref(nb)))
        return out[:nb.value].view(dtype)

    def spmv(self, x, y, cfg: Config | None = None, alpha=1.0, beta=0.0):
        """y = alpha A x + beta y on torch CUDA tensors (float64 or float32)."""
        import torch
        dtype = DTYPE_F64 if x.dtype == torch.float64 else DTYPE_F32
        assert y.dtype == x.dtype and x.is_cuda and y.is_cuda
        with self.ctx.ordered():
            _check(lib().cp_spmv(self.ctx.handle, self._h,
                                 byref(cfg) if cfg is not None else None, dtype, alpha, _ptr(x),
                                 beta, _ptr(y)))

    def predict(self):
        cfg = Config()
        ms = np.zeros(4, np.float32)
        _check(lib().cp_predict(self.ctx.handle, self._h, byref(cfg), _ptr(ms)))
        return cfg, ms

    def _solve(self, fn, b, x, opts: SolveOpts | None, force: Config | None, raise_on_error):
        o = opts if opts is not None else default_opts()
        if force is not None:
            o.force = ctypes.pointer(force)
        info = SolveInfo()
        with self.ctx.ordered():
            st = fn(self.ctx.handle, self._h, _ptr(b), _ptr(x), byref(o), byref(info))
        if raise_on_error:
            _check(st)
        return info

    def solve_cg(self, b, x, opts=None, force=None, raise_on_error=True) -> SolveInfo:
        """CG on torch CUDA float64 tensors b, x (x: x0 in, solution out)."""
        return self._solve(lib().cp_solve_cg, b, x, opts, force, raise_on_error)

    def solve_gmres(self, b, x, opts=None, force=None, raise_on_error=True) -> SolveInfo:
        """Restarted GMRES(m) on torch CUDA float64 tensors b, x."""
        return self._solve(lib().cp_solve_gmres, b, x, opts, force, raise_on_error)


class Server:
    """cp_server_*: continuous-batching solve server on a context's device."""

    def __init__(self, ctx: Context, **opts):
        self.ctx = ctx
        o = ServerOpts()
        lib().cp_server_opts_default(byref(o))
        for k, v in opts.items():
            _set_field(o, k, v)
        self.opts = o
        self._h = c_void_p()
        _check(lib().cp_server_create(ctx.handle, byref(o), byref(self._h)))
        self._keep = {}

    def submit(self, rid, mat: Matrix, solver, b, x):
        """Queue a solve; b and x (torch CUDA float64) must stay alive until polled.
        The lanes run on their own streams, so torch work that filled b and x is
        waited for here."""
        import torch
        torch.cuda.current_stream(self.ctx.device).synchronize()
        r = Request(rid, mat._h.value, solver, 0, b.data_ptr(), x.data_ptr())
        self._keep[rid] = (mat, b, x)
        _check(lib().cp_server_submit(self._h, byref(r)))

    def poll(self, capacity=4096):
        out = (Result * capacity)()
        cnt = c_int32()
        _check(lib().cp_server_poll(self._h, out, capacity, byref(cnt)))
        res = [out[i] for i in range(cnt.value)]
        for r in res:
            self._keep.pop(r.id, None)
        return res

    def drain(self, timeout_s=600.0):
        _check(lib().cp_server_drain(self._h, timeout_s))

    def close(self):
        if self._h:
            lib().cp_server_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
