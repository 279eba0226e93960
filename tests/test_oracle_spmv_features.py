"""Pins of the oracle's SpMV and Table IV features against brute force and closed forms."""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2411_10143_b300 import workloads as W

GOLD = Path(__file__).parent / "golden"


def dense(A):
    D = np.zeros((A.nrows, A.ncols))
    for i in range(A.nrows):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            D[i, A.col[k]] = A.val[k]
    return D


@pytest.mark.parametrize("shape", [(1, 1), (7, 5), (33, 40), (200, 200), (65, 3)])
def test_spmv_exact_integer_vs_dense(shape):
    n, m = shape
    rng = np.random.default_rng(n * 1000 + m)
    lens = rng.integers(0, min(m, 9) + 1, n)
    A = W.random_csr(n, m, lens, seed=n + m, int_values=True)
    x = W.int_vector(m, seed=5)
    # every summation order of small integers is exact: equality is required
    assert np.array_equal(oracle.spmv(A, x), dense(A) @ x)
    assert np.array_equal(oracle.spmv_f32(A, x).astype(np.float64), dense(A) @ x)


def test_spmv_random_float_vs_dense():
    A = W.random_csr(300, 250, np.random.default_rng(1).integers(0, 30, 300), seed=2)
    x = W.vector(250, 3)
    ref = dense(A) @ x
    assert np.linalg.norm(oracle.spmv(A, x) - ref) <= 1e-14 * np.linalg.norm(ref)


def test_spmv_empty():
    A = W.random_csr(4, 4, [0, 0, 0, 0], seed=0)
    assert np.array_equal(oracle.spmv(A, np.ones(4)), np.zeros(4))


# ------------------------------------------------------------------ features
def feat(A):
    return dict(zip(oracle.FEATURE_NAMES, oracle.features(A)))


def test_features_golden_hand_derived():
    g = json.loads((GOLD / "features_4x5.json").read_text())
    A = W.Matrix(g["nrows"], g["ncols"], np.array(g["rowptr"], np.int32),
                 np.array(g["col"], np.int32), np.ones(len(g["col"])))
    f = feat(A)
    for k, v in g["features"].items():
        assert f[k] == pytest.approx(v, rel=1e-15, abs=0), k


@pytest.mark.parametrize("N", [3, 4, 8, 31])
def test_features_poisson2d_closed_form(N):
    A = W.poisson2d(N)
    f = feat(A)
    n = N * N
    nnz = 5 * N * N - 4 * N
    assert f["nnz"] == nnz and f["max"] == 5 and f["min"] == 3
    assert f["ndiag"] == 5
    # row lengths: 4 corners of 3, 4(N-2) edge rows of 4, (N-2)^2 interior rows of 5
    lens = [3] * 4 + [4] * (4 * (N - 2)) + [5] * ((N - 2) ** 2)
    mean = nnz / n
    assert f["mean"] == pytest.approx(mean, rel=1e-15)
    assert f["sd"] == pytest.approx(math.sqrt(sum((l - mean) ** 2 for l in lens) / n), rel=1e-13)
    # c_last - c_first: 2N on interior grid rows, (1 or 0) + N on the first/last grid row
    width = 2 * N * N * (N - 2) + 2 * (N - 1 + N * N)
    assert f["distavg"] == pytest.approx(width / n, rel=1e-15)
    # longest consecutive run is the i-1, i, i+1 triple: 3 inside a grid row, 2 at its ends
    runs = N * (3 * (N - 2) + 4)
    assert f["clusteravg"] == pytest.approx(runs / n, rel=1e-15)
    assert f["fill"] == pytest.approx(n * f["max"] / nnz, rel=1e-15)
    assert f["diagfill"] == pytest.approx(n * 5 / nnz, rel=1e-15)
    assert f["density"] == pytest.approx(nnz / (n * n), rel=1e-15)


@pytest.mark.parametrize("N", [3, 6, 10])
def test_features_poisson3d_closed_form(N):
    f = feat(W.poisson3d(N))
    assert f["nnz"] == 7 * N**3 - 6 * N**2
    assert (f["max"], f["min"], f["ndiag"]) == (7, 4, 7)
    assert f["maxavg"] == pytest.approx(7 - (7 * N**3 - 6 * N**2) / N**3, rel=1e-14)


def test_features_identity():
    f = feat(W.diag_matrix(np.ones(50)))
    assert f["sd"] == 0 and f["cov"] == 0 and f["ndiag"] == 1
    assert f["fill"] == 1 and f["diagfill"] == 1 and f["distavg"] == 0
    assert f["clusteravg"] == 1 and f["max"] == 1 and f["min"] == 1


@pytest.mark.parametrize("k", [1, 2, 9])
def test_features_dense(k):
    f = feat(W.dense_matrix(k))
    assert f["ndiag"] == 2 * k - 1 and f["clusteravg"] == k and f["distavg"] == k - 1
    assert f["fill"] == 1 and f["diagfill"] == pytest.approx((2 * k - 1) / k)
    assert f["density"] == 1


def brute_features(A):
    """Independent brute force over Python lists (set for ndiag, numpy std for sd)."""
    rows = [list(A.col[A.rowptr[i]:A.rowptr[i + 1]]) for i in range(A.nrows)]
    lens = np.array([len(r) for r in rows], float)
    nnz = int(lens.sum())
    offs = {c - i for i, r in enumerate(rows) for c in r}

    def longest(r):
        best, cur = 0, 0
        for j, c in enumerate(r):
            cur = cur + 1 if j > 0 and c == r[j - 1] + 1 else 1
            best = max(best, cur)
        return best

    n = A.nrows
    mean = nnz / n
    sd = float(np.std(lens))
    return {
        "nrows": n, "ncols": A.ncols, "nnz": nnz, "density": nnz / (n * A.ncols),
        "mean": mean, "sd": sd, "cov": sd / mean if mean else 0.0,
        "max": lens.max(), "min": lens.min(), "maxavg": lens.max() - mean,
        "distavg": sum(r[-1] - r[0] for r in rows if r) / n,
        "clusteravg": sum(longest(r) for r in rows) / n,
        "fill": n * lens.max() / nnz if nnz else 0.0, "ndiag": len(offs),
        "diagfill": n * len(offs) / nnz if nnz else 0.0,
    }


@pytest.mark.parametrize("seed", range(6))
def test_features_bruteforce_random(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 60)), int(rng.integers(1, 70))
    lens = rng.integers(0, min(m, 12) + 1, n)
    if seed % 2:
        lens[rng.integers(0, n)] = m  # a full row
    A = W.random_csr(n, m, lens, seed=seed)
    f, g = feat(A), brute_features(A)
    for k in oracle.FEATURE_NAMES:
        assert f[k] == pytest.approx(g[k], rel=1e-12, abs=1e-15), k
