"""Host-side arithmetic of bench.py (no GPU): the algorithmic byte and FMA
counts behind the roofline fractions, and the guard that drops the recorded
DRAM traffic of the persistent CG kernel once its sources change."""
import numpy as np
import pytest

import bench
from paper_2411_10143_b300 import workloads as W


def test_spmv_bytes_count_every_array_once():
    """One definition for every configuration: values (8 B) and column indices
    (4 B) per non-zero, the row pointer, x read once and y written once.  The
    formats' own layouts are reported beside it: DIA drops the indices and the
    row pointer; COO carries a row index per non-zero instead of the row
    pointer; the others move what CSR moves."""
    A = W.random_csr(37, 41, [3, 0, 5, 1] * 9 + [2], seed=4)
    n, nc, nnz = A.nrows, A.ncols, A.nnz
    vals, cols, rowptr, x, y = 8 * nnz, 4 * nnz, 4 * (n + 1), 8 * nc, 8 * n
    assert bench.spmv_bytes(A) == vals + cols + rowptr + x + y
    assert bench.format_bytes(A, "ELL") == bench.spmv_bytes(A)
    assert bench.format_bytes(A, "HYB-K0") == bench.spmv_bytes(A)
    assert bench.format_bytes(A, "DIA") == vals + x + y
    assert bench.format_bytes(A, "COO") == vals + cols + 4 * nnz + x + y
    assert bench.cg_iteration_bytes(A) == vals + cols + rowptr + x + y + 9 * 8 * n
    assert bench.cg_iteration_bytes(A, "DIA") == vals + x + y + 9 * 8 * n


def test_gmres_fma_count_by_brute_force():
    """Step j of a cycle: nnz + (j + 1) n + (j + 1) n + n; a cycle of L steps adds
    L n (x += V y) and nnz + n (restart residual and its norm).  Several full
    cycles and a ragged last one."""
    n, nnz, m = 1000, 7000, 30
    for iters in (1, 29, 30, 31, 95):
        total, left = 0, iters
        while left > 0:
            L = min(m, left)
            for j in range(L):
                total += nnz + (j + 1) * n + (j + 1) * n + n
            total += L * n + nnz + n
            left -= L
        assert bench.gmres_dfma(n, nnz, iters, m) == total, iters


def test_recorded_traffic_only_for_its_sources(monkeypatch):
    A = W.poisson3d(4)
    rec = dict(bench.PERSIST_TRAFFIC, n=A.nrows, sha256=bench.persist_sources_sha256(),
               dram_bytes_per_iteration=1000.0)
    monkeypatch.setattr(bench, "PERSIST_TRAFFIC", rec)
    assert bench.persist_traffic(A, "DIA", 7) == pytest.approx(7000.0)
    assert bench.persist_traffic(A, "ELL", 7) is None  # another format's kernel
    assert bench.persist_traffic(W.poisson3d(5), "DIA", 7) is None  # another size
    monkeypatch.setattr(bench, "PERSIST_TRAFFIC", dict(rec, sha256="0" * 64))
    assert bench.persist_traffic(A, "DIA", 7) is None  # the sources changed since
