"""GPU SpMV family vs the oracle's CSR definition, element by element.

Integer-valued data makes every summation order exact, so every kernel must
match bit for bit; random FP64 data must agree within 1e-12 (norm-wise relative,
the tolerance the method's acceptance fixes for FP64 SpMV) and FP32 within 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_10143_b300 import cascade as C
from paper_2411_10143_b300 import workloads as W
from gpu_helpers import all_configs, ragged_matrices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = C.Context(0)
    yield c
    c.close()


def usable(A, cfgs):
    """Every configuration, except DIA where the matrix has more than 1024 diagonals
    (DIA refuses those with CP_ERR_FOOTPRINT, checked in the conversion tests)."""
    nd = len(oracle.to_dia(A)[0])
    return [c for c in cfgs if not (c.fmt == C.FMT_DIA and nd > 1024)]


def run(mat, cfg, x, dtype=torch.float64, alpha=1.0, beta=0.0, y0=None):
    xd = torch.as_tensor(x, dtype=dtype, device="cuda")
    yd = (torch.as_tensor(y0, dtype=dtype, device="cuda").clone() if y0 is not None
          else torch.full((mat.nrows,), float("nan"), dtype=dtype, device="cuda"))
    mat.spmv(xd, yd, cfg, alpha, beta)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("mi", range(8))
def test_spmv_integer_bit_exact(ctx, mi):
    A = ragged_matrices(True)[mi]
    M = ctx.load(A)
    x = W.int_vector(A.ncols, 7)
    ref = oracle.spmv(A, x)
    for cfg in usable(A, all_configs()):
        y = run(M, cfg, x)
        assert np.array_equal(y, ref), repr(cfg)
        y32 = run(M, cfg, x, torch.float32)
        assert np.array_equal(y32.astype(np.float64), ref), repr(cfg)


@pytest.mark.parametrize("mi", range(8))
def test_spmv_random_fp64_and_fp32(ctx, mi):
    A = ragged_matrices(False)[mi]
    M = ctx.load(A)
    x = W.vector(A.ncols, 5)
    ref = oracle.spmv(A, x)
    ref32 = oracle.spmv_f32(A, x).astype(np.float64)
    nr = max(np.linalg.norm(ref), 1e-300)
    for cfg in usable(A, all_configs()):
        y = run(M, cfg, x)
        assert np.linalg.norm(y - ref) <= 1e-12 * nr, repr(cfg)
        y32 = run(M, cfg, x, torch.float32).astype(np.float64)
        assert np.linalg.norm(y32 - ref32) <= 1e-5 * max(np.linalg.norm(ref32), 1e-30), repr(cfg)


@pytest.mark.parametrize("alpha,beta", [(0.5, -2.0), (0.5, 0.0), (1.0, 3.0)])
def test_spmv_general_alpha_beta(ctx, alpha, beta):
    """y = alpha A x + beta y0 in every configuration: the general form, a scaled
    product over a zero y, and alpha = 1 over a nonzero y (the COO kernel's
    alpha = 1 variants add with atomics)."""
    A = ragged_matrices(False)[2]
    M = ctx.load(A)
    x = W.vector(A.ncols, 1)
    y0 = W.vector(A.nrows, 2)
    ref = alpha * oracle.spmv(A, x) + beta * y0
    for cfg in usable(A, all_configs()):
        y = run(M, cfg, x, alpha=alpha, beta=beta, y0=y0)
        assert np.linalg.norm(y - ref) <= 1e-12 * np.linalg.norm(ref), repr(cfg)


def test_rejects_invalid_csr(ctx):
    A = W.random_csr(10, 10, [2] * 10, seed=0)
    bad = A.col.copy()
    bad[3] = 99
    with pytest.raises(C.CascadeError) as e:
        ctx.csr_load(10, 10, A.rowptr, bad, A.val)
    assert e.value.status == C.ERR_INVALID
    rp = A.rowptr.copy()
    rp[5] = rp[6] + 1
    with pytest.raises(C.CascadeError):
        ctx.csr_load(10, 10, rp, A.col, A.val)
    unsorted = A.col.copy()
    unsorted[0], unsorted[1] = unsorted[1], unsorted[0]
    with pytest.raises(C.CascadeError):
        ctx.csr_load(10, 10, A.rowptr, unsorted, A.val)


def test_unsupported_config(ctx):
    M = ctx.load(W.poisson2d(8))
    x = torch.ones(64, dtype=torch.float64, device="cuda")
    y = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(C.CascadeError) as e:
        M.spmv(x, y, C.config("CSR", C.ALGO_VECTOR, tpv=3))
    assert e.value.status == C.ERR_UNSUPPORTED
    with pytest.raises(C.CascadeError):
        M.spmv(x, y, C.config("SELL", sigma=48 + 1))


def test_footprint_refusal(ctx):
    A = W.powerlaw(4000, lmax=3000, seed=3)
    M = ctx.load(A)
    ctx.set_format_budget(1 << 20)
    try:
        with pytest.raises(C.CascadeError) as e:
            M.convert(C.config("ELL"))
        assert e.value.status == C.ERR_FOOTPRINT
    finally:
        ctx.set_format_budget(4 << 30)
