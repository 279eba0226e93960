"""The synthetic inputs follow their stated recipes (no GPU): stencil values and
sizes, the convection-diffusion rows, the SPD power law's symmetry and strict
diagonal dominance, the banded offsets and fill, the power law's mean and
longest row, and the uniform matrix's row lengths.  Every matrix is valid CSR
(sorted unique columns in range)."""
import numpy as np
import pytest

from paper_2411_10143_b300 import workloads as W


def dense(A):
    D = np.zeros((A.nrows, A.ncols))
    for i in range(A.nrows):
        for k in range(A.rowptr[i], A.rowptr[i + 1]):
            D[i, A.col[k]] += A.val[k]
    return D


def valid_csr(A):
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.nnz == A.col.size == A.val.size
    assert np.all(np.diff(A.rowptr) >= 0)
    assert A.col.min(initial=0) >= 0 and A.col.max(initial=0) < A.ncols
    for i in range(A.nrows):
        c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0), i


@pytest.mark.parametrize("k", [3, 6])
def test_poisson_stencils(k):
    A2, A3 = W.poisson2d(k), W.poisson3d(k)
    valid_csr(A2)
    valid_csr(A3)
    assert A2.nrows == k * k and A2.nnz == 5 * k * k - 4 * k
    assert A3.nrows == k ** 3 and A3.nnz == 7 * k ** 3 - 6 * k * k
    D2, D3 = dense(A2), dense(A3)
    assert np.array_equal(D2, D2.T) and np.array_equal(D3, D3.T)
    assert np.all(np.diag(D2) == 4.0) and np.all(np.diag(D3) == 6.0)
    for D in (D2, D3):
        off = D - np.diag(np.diag(D))
        assert set(np.unique(off)) <= {0.0, -1.0}
    # the 1D second difference along x in the 3D ordering: index i and i + 1
    assert D3[0, 1] == -1.0 and D3[k - 1, k] == 0.0  # no wrap between grid lines


def test_convection_diffusion_rows():
    """Pe = 10 per axis, scaled by h^2: diagonal 66, upwind -21, downwind -1."""
    k = 5
    A = W.convdiff3d(k)
    valid_csr(A)
    D = dense(A)
    c = (2 * k + 2) * k + 2  # the centre point (2, 2, 2)
    row = D[c]
    assert row[c] == 66.0
    for s in (1, k, k * k):
        assert row[c - s] == -21.0 and row[c + s] == -1.0
    assert np.count_nonzero(row) == 7
    assert not np.array_equal(D, D.T)
    # irreducibly diagonally dominant: |d_i| >= sum of the others, strictly somewhere
    offsum = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    assert np.all(np.abs(np.diag(D)) >= offsum) and np.any(np.abs(np.diag(D)) > offsum)


def test_spd_power_law_is_symmetric_and_dominant():
    A = W.spd_powerlaw(600, seed=9)
    valid_csr(A)
    D = dense(A)
    assert np.allclose(D, D.T, rtol=0, atol=0)
    offsum = np.abs(D).sum(axis=1) - np.abs(np.diag(D))
    assert np.allclose(np.diag(D), offsum + 1.0)
    assert np.linalg.eigvalsh(D).min() >= 1.0 - 1e-9  # Gershgorin
    assert np.all(np.abs(D - np.diag(np.diag(D))) <= 2.0)  # two U[-1,1] draws at most


def test_banded_offsets_and_fill():
    n = 3000
    A = W.banded(n, 64, 0.6, seed=5)
    valid_csr(A)
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    off = A.col - rows
    assert off.min() >= -32 and off.max() <= 31
    assert np.count_nonzero(off == 0) == n  # the diagonal in every row
    inner = (rows >= 32) & (rows < n - 32)  # rows whose 64 band slots are all in range
    share = np.count_nonzero(inner & (off != 0)) / (63 * (n - 64))
    assert abs(share - 0.6) < 0.02


def test_power_law_mean_and_longest_row():
    n, lmax = 20000, 1000
    A = W.powerlaw(n, lmax=lmax, seed=11)
    valid_csr(A)
    lens = np.diff(A.rowptr)
    # one row drawn at lmax entries; its duplicate column draws are merged
    assert lens.min() >= 1 and 0.95 * lmax <= lens.max() <= lmax
    assert abs(lens.mean() - 16.0) < 1.0  # rescaled to the mean (duplicates merged)
    assert np.median(lens) < lens.mean() / 2  # heavy tail


def test_uniform_rows():
    A = W.uniform_random(5000, 8, seed=3)
    valid_csr(A)
    lens = np.diff(A.rowptr)
    assert lens.max() == 8 and lens.mean() > 7.99  # rare duplicate draws merged


def test_request_stream_mix_sizes_and_arrivals():
    """Serving requests: Poisson arrivals at the given rate, n log-uniform in
    [1e3, 1e6], 40 % Poisson (2D and 3D half each), 30 % SPD power law, 30 %
    convection-diffusion; a request's system has about n rows."""
    reqs = W.request_stream(4000, rate_per_s=50.0, seed=3000)
    kinds = np.array([r.kind for r in reqs])
    share = {k: np.mean(kinds == k) for k in ("poisson2d", "poisson3d", "spd_powerlaw", "convdiff")}
    assert abs(share["poisson2d"] + share["poisson3d"] - 0.4) < 0.03
    assert abs(share["poisson2d"] - share["poisson3d"]) < 0.04
    assert abs(share["spd_powerlaw"] - 0.3) < 0.03 and abs(share["convdiff"] - 0.3) < 0.03
    n = np.array([r.n for r in reqs])
    assert n.min() >= 1000 and n.max() <= 1_000_000
    logn = np.log10(n)
    assert abs(np.median(logn) - 4.5) < 0.1  # the middle of [3, 6] on a log scale
    assert abs(np.mean((logn >= 3.0) & (logn < 4.0)) - 1 / 3) < 0.03
    t = np.array([r.arrival_s for r in reqs])
    gaps = np.diff(t)
    assert np.all(gaps > 0) and abs(gaps.mean() * 50.0 - 1.0) < 0.05
    assert abs(np.std(gaps) / np.mean(gaps) - 1.0) < 0.1  # exponential gaps
    for r in reqs[:12]:
        A = W.request_matrix(r) if r.n < 30000 else None
        if A is not None:
            assert 0.5 * r.n <= A.nrows <= 2.0 * r.n, (r.kind, r.n, A.nrows)


def test_spd_variant_is_symmetric_and_strictly_dominant():
    import scipy.sparse as sp
    A = W.powerlaw(3000, 1.8, 10.0, 400, 3)
    S = W.spd_variant(A)
    Ss = sp.csr_matrix((S.val, S.col, S.rowptr), shape=(S.nrows, S.ncols))
    assert abs(Ss - Ss.T).max() == 0
    diag = Ss.diagonal()
    off = np.asarray(abs(Ss).sum(1)).ravel() - np.abs(diag)
    assert np.allclose(diag, off + 1.0, rtol=1e-13, atol=0)  # sums in another order
    # the off-diagonal pattern is that of A + A^T
    As = sp.csr_matrix((np.ones(A.nnz), A.col, A.rowptr), shape=(A.nrows, A.ncols))
    As.setdiag(0)
    As.eliminate_zeros()
    pa = ((As + As.T) != 0).astype(np.int8)
    Sp = sp.csr_matrix((np.ones(S.nnz), S.col, S.rowptr), shape=(S.nrows, S.ncols))
    Sp.setdiag(0)
    Sp.eliminate_zeros()
    assert (pa != (Sp != 0).astype(np.int8)).nnz == 0


def test_batch_suite_sizes_and_families():
    suite = W.batch_suite(count=12)
    fams = [name.split("_")[0] for name, _ in suite]
    assert fams[:6] == ["p2d", "p3d", "pl", "uni", "band", "bimodal"]
    for name, make in suite[:6]:
        A = make()
        assert 2 ** 9 <= A.nrows <= 2 ** 15 + 2000, (name, A.nrows)
        assert A.nrows == A.ncols
