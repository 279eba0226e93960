"""GPU format conversions and Table IV features vs the oracle.

Conversions are integer work that copies values: every array must equal the
oracle's canonical layout bit for bit.  Integer-valued features must be equal;
the FP64 derived ones agree to 1e-12 (the GPU takes sd from exact integer
sums, the oracle sums (mean - r_i)^2 row by row)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_10143_b300 import cascade as C
from paper_2411_10143_b300 import workloads as W
from gpu_helpers import ragged_matrices

pytestmark = pytest.mark.gpu


def hyb_auto_width(A):
    """HYB's width for hyb_k = 0 as the header defines it: the smallest K >= 1 that
    at most a quarter of the rows exceed, else ceil(mean row length) when that
    is 1,023 or more."""
    lens = np.diff(A.rowptr)
    for K in range(1, 1023):
        if 4 * np.count_nonzero(lens > K) <= A.nrows:
            return K
    return max(1, -(-A.nnz // A.nrows))


@pytest.fixture(scope="module")
def ctx():
    c = C.Context(0)
    yield c
    c.close()


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint8)


@pytest.mark.parametrize("mi", range(8))
def test_conversions_bit_exact(ctx, mi):
    A = ragged_matrices(False)[mi]
    M = ctx.load(A)
    row, _, _ = oracle.to_coo(A)
    assert np.array_equal(M.format_export(C.config("COO"), "COO_ROW", np.int32), row)
    K, ld, ecol, eval_ = oracle.to_ell(A)
    cfg = C.config("ELL")
    assert M.format_dims(cfg)[:2] == [K, ld]
    assert np.array_equal(M.format_export(cfg, "ELL_COL", np.int32), ecol)
    assert np.array_equal(bits(M.format_export(cfg, "ELL_VAL", np.float64)), bits(eval_))
    for sigma in C.SIGMA_CLASSES:
        perm, clen, cptr, scol, sval = oracle.to_sell(A, 32, sigma)
        cfg = C.config("SELL", sigma=sigma)
        assert np.array_equal(M.format_export(cfg, "SELL_PERM", np.int32), perm), sigma
        assert np.array_equal(M.format_export(cfg, "SELL_CHUNK_LEN", np.int32), clen), sigma
        assert np.array_equal(M.format_export(cfg, "SELL_CHUNK_PTR", np.int64), cptr), sigma
        assert np.array_equal(M.format_export(cfg, "SELL_COL", np.int32), scol), sigma
        assert np.array_equal(bits(M.format_export(cfg, "SELL_VAL", np.float64)), bits(sval))
    for hk in (0, 1, 3):
        Kh = hk if hk > 0 else hyb_auto_width(A)
        ld, ec, ev, cr, cc, cv = oracle.to_hyb(A, Kh)
        cfg = C.config("HYB", hyb_k=hk)
        assert M.format_dims(cfg)[:3] == [Kh, ld, len(cr)]
        assert np.array_equal(M.format_export(cfg, "HYB_ELL_COL", np.int32), ec)
        assert np.array_equal(bits(M.format_export(cfg, "HYB_ELL_VAL", np.float64)), bits(ev))
        assert np.array_equal(M.format_export(cfg, "HYB_COO_ROW", np.int32), cr)
        assert np.array_equal(M.format_export(cfg, "HYB_COO_COL", np.int32), cc)
        assert np.array_equal(bits(M.format_export(cfg, "HYB_COO_VAL", np.float64)), bits(cv))
    offs, data = oracle.to_dia(A)
    cfg = C.config("DIA")
    if len(offs) <= 1024:
        assert M.format_dims(cfg)[:2] == [len(offs), A.nrows]
        assert np.array_equal(M.format_export(cfg, "DIA_OFFSETS", np.int32), offs)
        assert np.array_equal(bits(M.format_export(cfg, "DIA_VAL", np.float64)), bits(data))
    else:
        with pytest.raises(C.CascadeError) as e:
            M.convert(cfg)
        assert e.value.status == C.ERR_FOOTPRINT


INT_FEATURES = ("nrows", "ncols", "nnz", "max", "min", "ndiag")


def check_features(g, o):
    for k, name in enumerate(oracle.FEATURE_NAMES):
        if name in INT_FEATURES:
            assert g[k] == o[k], name
        else:
            assert g[k] == pytest.approx(o[k], rel=1e-12, abs=1e-300), name


@pytest.mark.parametrize("mi", range(8))
def test_features_vs_oracle(ctx, mi):
    A = ragged_matrices(False)[mi]
    check_features(ctx.load(A).features(), oracle.features(A))


def test_features_long_rows_and_structures(ctx):
    mats = [W.powerlaw(30000, lmax=5000, seed=4), W.poisson2d(64), W.poisson3d(16),
            W.banded(20000, 64, 0.6, seed=2), W.dense_matrix(70), W.diag_matrix(np.ones(33)),
            W.uniform_random(5000, 8, seed=3, ncols=7000)]
    for A in mats:
        check_features(ctx.load(A).features(), oracle.features(A))


@pytest.mark.parametrize("k,lens", [(1100, None), (4000, "skewed")])
def test_hyb_default_width_rule(ctx, k, lens):
    """hyb_k = 0: the 75th percentile of the row lengths, and ceil(mean) when that
    lies past the 1,023-entry histogram (a dense 1,100 x 1,100 matrix); the
    layout equals the oracle's at that width and the SpMV agrees."""
    if lens is None:
        A = W.dense_matrix(k, seed=3)
    else:
        A = W.random_csr(k, k, [1, 2, 2, 3, 40] * (k // 5), seed=6)
    K = hyb_auto_width(A)
    assert K == (k if lens is None else 3)
    M = ctx.load(A)
    cfg = C.config("HYB")
    ld, ec, ev, cr, cc, cv = oracle.to_hyb(A, K)
    assert M.format_dims(cfg)[:3] == [K, ld, len(cr)]
    assert np.array_equal(M.format_export(cfg, "HYB_ELL_COL", np.int32), ec)
    assert np.array_equal(M.format_export(cfg, "HYB_COO_ROW", np.int32), cr)
    x = W.vector(A.ncols, 2)
    ref = oracle.spmv(A, x)
    xd = torch.as_tensor(x, device="cuda")
    yd = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    M.spmv(xd, yd, cfg)
    torch.cuda.synchronize()
    assert np.linalg.norm(yd.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
