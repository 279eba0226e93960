"""Pins of the oracle's canonical format layouts: hand-derived layouts and round trips."""
import json
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2411_10143_b300 import workloads as W

GOLD = json.loads((Path(__file__).parent / "golden" / "formats_5x6.json").read_text())


def gold_matrix():
    return W.Matrix(GOLD["nrows"], GOLD["ncols"], np.array(GOLD["rowptr"], np.int32),
                    np.array(GOLD["col"], np.int32), np.array(GOLD["val"], np.float64))


def same_csr(A, B):
    return (np.array_equal(A.rowptr, B.rowptr) and np.array_equal(A.col, B.col)
            and np.array_equal(A.val.view(np.int64), B.val.view(np.int64)))


def test_coo_golden():
    row, col, val = oracle.to_coo(gold_matrix())
    assert row.tolist() == GOLD["coo_row"]
    assert col.tolist() == GOLD["col"] and val.tolist() == GOLD["val"]


def test_ell_golden():
    K, ld, ecol, eval_ = oracle.to_ell(gold_matrix())
    g = GOLD["ell"]
    assert (K, ld) == (g["K"], g["ld"])
    c, v = ecol.reshape(K, ld), eval_.reshape(K, ld)
    assert c[:, :5].tolist() == g["col_first5"] and v[:, :5].tolist() == g["val_first5"]
    assert (c[:, 5:] == -1).all() and (v[:, 5:] == 0).all()


@pytest.mark.parametrize("key,C,sigma", [("sell_C2_s4", 2, 4), ("sell_C2_s1", 2, 1)])
def test_sell_golden(key, C, sigma):
    perm, clen, cptr, scol, sval = oracle.to_sell(gold_matrix(), C, sigma)
    g = GOLD[key]
    assert perm.tolist() == g["perm"] and clen.tolist() == g["chunk_len"]
    assert cptr.tolist() == g["chunk_ptr"]
    assert scol.tolist() == g["col"] and sval.tolist() == g["val"]


def test_hyb_golden():
    ld, ecol, eval_, crow, ccol, cval = oracle.to_hyb(gold_matrix(), 1)
    g = GOLD["hyb_K1"]
    assert ecol[:5].tolist() == g["ell_col_first5"] and eval_[:5].tolist() == g["ell_val_first5"]
    assert crow.tolist() == g["coo_row"] and ccol.tolist() == g["coo_col"]
    assert cval.tolist() == g["coo_val"]


def rand_matrix(seed, n=None):
    rng = np.random.default_rng(seed)
    n = n or int(rng.integers(1, 300))
    m = int(rng.integers(1, 400))
    lens = rng.integers(0, min(m, 20) + 1, n)
    lens[rng.random(n) < 0.1] = 0
    if n > 3:
        lens[rng.integers(0, n)] = min(m, 150)
    return W.random_csr(n, m, lens, seed=seed)


@pytest.mark.parametrize("seed", range(8))
def test_round_trips(seed):
    A = rand_matrix(seed)
    n, m, nnz = A.nrows, A.ncols, A.nnz
    row, col, val = oracle.to_coo(A)
    assert same_csr(oracle.coo_to_csr(n, m, row, col, val), A)
    K, ld, ecol, eval_ = oracle.to_ell(A)
    assert same_csr(oracle.ell_to_csr(n, m, K, ld, ecol, eval_, nnz), A)
    for C, sigma in [(32, 1), (32, 32), (8, 64), (16, 1024), (4, 3)]:
        perm, clen, cptr, scol, sval = oracle.to_sell(A, C, sigma)
        assert sorted(perm.tolist()) == list(range(n))
        lens = np.diff(A.rowptr)[perm]
        for w0 in range(0, n, sigma):  # longest first inside each window, stable ties
            seg = lens[w0:w0 + sigma]
            assert (np.diff(seg) <= 0).all()
            p = perm[w0:w0 + sigma]
            for a in range(len(seg) - 1):
                if seg[a] == seg[a + 1]:
                    assert p[a] < p[a + 1]
        assert same_csr(oracle.sell_to_csr(n, m, C, perm, clen, cptr, scol, sval, nnz), A)
    for Kh in (0, 1, 3, 8, 1000):
        ld, ec, ev, cr, cc, cv = oracle.to_hyb(A, Kh)
        assert same_csr(oracle.hyb_to_csr(n, m, Kh, ld, ec, ev, cr, cc, cv, nnz), A)


def test_padding_and_spmv_consistency():
    """SpMV recomputed from each layout by its own definition equals CSR SpMV exactly
    (integer data: every order exact)."""
    A = W.random_csr(97, 80, np.random.default_rng(3).integers(0, 12, 97), seed=4,
                     int_values=True)
    x = W.int_vector(80, 1)
    y = oracle.spmv(A, x)
    K, ld, ecol, eval_ = oracle.to_ell(A)
    c, v = ecol.reshape(K, ld), eval_.reshape(K, ld)
    ye = np.array([sum(v[k, i] * x[c[k, i]] for k in range(K) if c[k, i] >= 0)
                   for i in range(A.nrows)])
    assert np.array_equal(ye, y)
    perm, clen, cptr, scol, sval = oracle.to_sell(A, 8, 16)
    ys = np.zeros(A.nrows)
    for s in range(A.nrows):
        ch, r = divmod(s, 8)
        for k in range(clen[ch]):
            j = cptr[ch] + k * 8 + r
            if scol[j] >= 0:
                ys[perm[s]] += sval[j] * x[scol[j]]
    assert np.array_equal(ys, y)


def test_dia_golden():
    offs, data = oracle.to_dia(gold_matrix())
    assert offs.tolist() == GOLD["dia"]["offsets"]
    assert data.reshape(len(offs), GOLD["nrows"]).tolist() == GOLD["dia"]["data"]


@pytest.mark.parametrize("seed", range(4))
def test_dia_spmv_consistency(seed):
    """y_i = sum_d data[d][i] x[i + off_d] equals CSR SpMV exactly on integer data."""
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 120)), int(rng.integers(1, 140))
    A = W.random_csr(n, m, rng.integers(0, 9, n), seed=seed, int_values=True)
    x = W.int_vector(m, seed)
    offs, data = oracle.to_dia(A)
    D = data.reshape(len(offs), n)
    y = np.zeros(n)
    for d, o in enumerate(offs):
        for i in range(n):
            if 0 <= i + o < m:
                y[i] += D[d, i] * x[i + o]
    assert np.array_equal(y, oracle.spmv(A, x))
    # every stored value appears exactly once
    assert np.count_nonzero(D) == np.count_nonzero(A.val)
