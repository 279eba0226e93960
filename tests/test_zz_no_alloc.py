"""The allocation-free SpMV entry point (cp_spmv_csr_merge_noalloc).

Some callers cannot allocate device memory where they need an SpMV (their
device memory is owned by an arena, or allocating would synchronise a stream
they are capturing or a callback they run in), so they cannot create a context
or a matrix handle.  This entry point takes plain device pointers and keeps its
scratch in a fixed library array.  The test checks it, through the C ABI,
against the existing cp_spmv with the same merge-path configuration, within the
FP64 SpMV tolerance of the other tests (1e-12 relative), on two calls in a row
with different matrices, so a stale carry left by the first call would show.
Both calls are also compared with the oracle's CSR SpMV on the same inputs.
It sits in a file pytest collects last."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_10143_b300 import cascade as C
from paper_2411_10143_b300 import workloads as W

pytestmark = pytest.mark.gpu


def reference_and_noalloc(ctx, A, seed):
    M = ctx.load(A)
    x = torch.as_tensor(W.vector(A.ncols, seed), device="cuda")
    y_ref = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    M.spmv(x, y_ref, C.config("CSR", C.ALGO_MERGE))
    rp = torch.as_tensor(A.rowptr, device="cuda")
    ci = torch.as_tensor(A.col, device="cuda")
    va = torch.as_tensor(A.val, device="cuda")
    y = torch.full((A.nrows,), float("nan"), dtype=torch.float64, device="cuda")
    C.spmv_csr_merge_noalloc(A.nrows, A.ncols, rp, ci, va, x, y)
    torch.cuda.synchronize()
    return y_ref.cpu().numpy(), y.cpu().numpy()


def test_noalloc_matches_cp_spmv_on_two_calls_in_a_row():
    ctx = C.Context(0)
    rng = np.random.default_rng(11)
    first = W.powerlaw(60000, lmax=20000, seed=5)          # ~550 tiles, one very long row
    lens = rng.integers(0, 12, 3001)
    second = W.random_csr(3001, 2500, lens, seed=6)         # a few tiles, ragged tail
    for A, seed in ((first, 1), (second, 2)):
        ref, got = reference_and_noalloc(ctx, A, seed)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        exact = oracle.spmv(A, W.vector(A.ncols, seed))
        assert np.linalg.norm(got - exact) <= 1e-12 * np.linalg.norm(exact)
    ctx.close()


def test_noalloc_setup_call_on_an_empty_row():
    """The one-time set-up can be done by a 1-row, nnz = 0 call (y = 0)."""
    rp = torch.zeros(2, dtype=torch.int32, device="cuda")
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    v = torch.empty(0, dtype=torch.float64, device="cuda")
    x = torch.ones(1, dtype=torch.float64, device="cuda")
    y = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    C.spmv_csr_merge_noalloc(1, 1, rp, e, v, x, y)
    torch.cuda.synchronize()
    assert y.item() == 0.0


def test_noalloc_binding_checks_arrays_before_the_call():
    """Wrong dtypes or arrays shorter than their sizes never reach the kernel."""
    A = W.random_csr(40, 30, np.full(40, 3), seed=3)
    rp = torch.as_tensor(A.rowptr, device="cuda")
    ci = torch.as_tensor(A.col, device="cuda")
    va = torch.as_tensor(A.val, device="cuda")
    x = torch.zeros(A.ncols, dtype=torch.float64, device="cuda")
    y = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    bad = [dict(rowptr=rp.long()), dict(col=ci.long()), dict(x=x.float()), dict(val=va.cpu()),
           dict(x=x[:-1]), dict(y=y[:-1]), dict(rowptr=rp[:-1]), dict(nnz=A.nnz + 1)]
    for b in bad:
        args = dict(rowptr=rp, col=ci, val=va, x=x, y=y)
        args.update(b)
        with pytest.raises(C.CascadeError) as e:
            C.spmv_csr_merge_noalloc(A.nrows, A.ncols, **args)
        assert e.value.status == C.ERR_INVALID


def test_noalloc_rejects_sizes_beyond_its_scratch():
    big = 65536 * 1792  # merge items the fixed scratch covers
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    i = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(C.CascadeError) as e:
        C.lib()  # status and message come back through the C ABI
        st = C.lib().cp_spmv_csr_merge_noalloc(big, 10, 10, C._ptr(i), C._ptr(i), C._ptr(d),
                                               C._ptr(d), C._ptr(d), None)
        C._check(st)
    assert e.value.status == C.ERR_INVALID and "maximum" in str(e.value)
