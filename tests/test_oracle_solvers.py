"""Pins of the oracle's CG, GMRES(m) and FP32-inner iterative refinement.

Each pin is fixed by mathematics, not by the oracle itself: finite termination
in exact arithmetic, the closed-form Poisson spectrum recovered from CG's
Lanczos coefficients, dense LU solutions, GMRES's minimal-residual property.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_10143_b300 import workloads as W


def dense(A):
    D = np.zeros((A.nrows, A.ncols))
    for i in range(A.nrows):
        D[i, A.col[A.rowptr[i]:A.rowptr[i + 1]]] = A.val[A.rowptr[i]:A.rowptr[i + 1]]
    return D


def from_dense(D):
    n = D.shape[0]
    r, c = np.nonzero(D)
    return W._from_rows_cols(n, D.shape[1], r, c, D[r, c], "dense")


# ------------------------------------------------------------------------ CG
def test_cg_identity_one_step():
    A = W.diag_matrix(np.ones(40))
    b = W.vector(40, 1)
    r = oracle.cg(A, b, tol=1e-14)
    assert r.iters == 1 and np.array_equal(r.x, b) and r.status == 0


@pytest.mark.parametrize("k", [2, 3, 5, 8])
def test_cg_k_distinct_eigenvalues(k):
    rng = np.random.default_rng(k)
    eig = np.sort(rng.uniform(1, 10, k))
    d = eig[rng.integers(0, k, 200)]
    d[:k] = eig  # every eigenvalue present
    A = W.diag_matrix(d)
    b = W.vector(200, k)
    r = oracle.cg(A, b, tol=1e-10)
    assert r.status == 0 and r.relres_true <= 1e-10
    assert r.iters <= k + 1  # k in exact arithmetic, one step of rounding slack
    assert np.allclose(r.x, b / d, rtol=1e-9)


@pytest.mark.parametrize("N", [12, 20])
def test_cg_lanczos_ritz_matches_poisson_spectrum(N):
    """T_jj = 1/a_j + b_{j-1}/a_{j-1}, T_{j,j+1} = sqrt(b_j)/a_j (Lanczos from CG);
    its extreme eigenvalues converge to 4 - 2cos(j pi/(N+1)) - 2cos(k pi/(N+1))."""
    A = W.poisson2d(N)
    b = W.vector(N * N, 7)
    r = oracle.cg(A, b, tol=1e-14, hist_cap=100000)
    a, be = r.alphas, r.betas
    m = len(a)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1 / a[j] + (be[j - 1] / a[j - 1] if j else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(be[j]) / a[j]
    ritz = np.linalg.eigvalsh(T)
    t = np.arange(1, N + 1) * math.pi / (N + 1)
    lam = (4 - 2 * np.cos(t)[:, None] - 2 * np.cos(t)[None, :]).ravel()
    assert ritz[0] == pytest.approx(lam.min(), rel=1e-8)
    assert ritz[-1] == pytest.approx(lam.max(), rel=1e-8)


def test_cg_matches_dense_solve_spd():
    A = W.spd_powerlaw(400, seed=5)
    xs = W.vector(400, 6)
    b = dense(A) @ xs
    r = oracle.cg(A, b, tol=1e-12)
    ref = np.linalg.solve(dense(A), b)
    assert r.relres_true <= 1e-12
    assert np.linalg.norm(r.x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_cg_all_core_build_solves_the_same_system():
    """The all-core timing build (the same source with -fopenmp) reaches the
    tolerance and the dense solution; only its reductions' rounding differs."""
    A = W.poisson3d(12)
    xs = W.vector(A.nrows, 7)
    b = oracle.spmv(A, xs)
    r1 = oracle.cg(A, b, tol=1e-10)
    rn = oracle.cg_all_cores(A, b, tol=1e-10)
    assert rn.status == 0 and rn.relres_true <= 1e-10 and rn.threads >= 1
    assert abs(rn.iters - r1.iters) <= 2
    assert np.linalg.norm(rn.x - xs) <= 1e-7 * np.linalg.norm(xs)


def test_cg_edge_cases():
    A = W.poisson2d(6)
    r = oracle.cg(A, np.zeros(36))
    assert r.iters == 0 and not r.x.any()
    r = oracle.cg(A, W.vector(36, 1), maxit=2, tol=1e-12)
    assert r.status == 4 and r.iters == 2
    neg = W.Matrix(A.nrows, A.ncols, A.rowptr, A.col, -A.val)
    assert oracle.cg(neg, W.vector(36, 1)).status == 5
    x0 = W.vector(36, 9)
    r = oracle.cg(A, W.vector(36, 1), x0=x0)
    assert r.relres_true <= 1e-10


# ------------------------------------------------------------------------ GMRES
@pytest.mark.parametrize("m", [5, 30])
def test_gmres_matches_dense_solve(m):
    A = W.convdiff3d(5)
    b = W.vector(A.nrows, 3)
    r = oracle.gmres(A, b, m=m, tol=1e-12)
    ref = np.linalg.solve(dense(A), b)
    assert r.status == 0 and r.relres_true <= 1e-12
    assert np.linalg.norm(r.x - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("k", [2, 4, 7])
def test_gmres_finite_termination_nonsymmetric(k):
    """A = S diag(lam) S^-1 with k distinct eigenvalues: full GMRES ends in <= k steps."""
    n = 30
    rng = np.random.default_rng(k)
    lam = rng.uniform(1, 5, k)[rng.integers(0, k, n)]
    S = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    D = S @ np.diag(lam) @ np.linalg.inv(S)
    A = from_dense(D)
    b = W.vector(n, k)
    r = oracle.gmres(A, b, m=n, tol=1e-9)
    assert r.status == 0 and r.iters <= k + 1


def test_gmres_residual_monotone_within_cycle():
    A = W.convdiff3d(6)
    b = W.vector(A.nrows, 2)
    m = 10
    r = oracle.gmres(A, b, m=m, tol=1e-10, hist_cap=10000)
    h = r.res_hist
    for c0 in range(0, len(h), m):
        seg = h[c0:c0 + m]
        assert (np.diff(seg) <= 1e-15).all()


@pytest.mark.parametrize("k", [3, 8, 15])
def test_gmres_residual_not_above_cg_on_spd(k):
    """Same Krylov space, GMRES minimises the residual norm: ||r_gmres_k|| <= ||r_cg_k||."""
    A = W.poisson2d(10)
    b = W.vector(100, 4)
    D = dense(A)
    xg = oracle.gmres(A, b, m=50, maxit=k, tol=1e-16).x
    xc = oracle.cg(A, b, maxit=k, tol=1e-16).x
    rg = np.linalg.norm(b - D @ xg)
    rc = np.linalg.norm(b - D @ xc)
    assert rg <= rc * (1 + 1e-10)


def test_gmres_full_equals_long_restart():
    A = from_dense(np.eye(12) * 3 + np.triu(np.ones((12, 12)), 1) * 0.5)
    b = W.vector(12, 1)
    r = oracle.gmres(A, b, m=12, tol=1e-13)
    assert r.iters <= 12 and r.relres_true <= 1e-13


def test_gmres_edge_cases():
    A = W.convdiff3d(4)
    r = oracle.gmres(A, np.zeros(A.nrows))
    assert r.iters == 0 and not r.x.any()
    r = oracle.gmres(A, W.vector(A.nrows, 1), maxit=3, tol=1e-14)
    assert r.status == 4 and r.iters == 3


# ------------------------------------------------------------------------ IR
@pytest.mark.parametrize("solver,make", [("cg", lambda: W.poisson3d(8)),
                                         ("gmres", lambda: W.convdiff3d(8)),
                                         ("cg", lambda: W.spd_powerlaw(2000, seed=3))])
def test_ir_reaches_fp64_residual(solver, make):
    A = make()
    b = W.vector(A.nrows, 11)
    r = oracle.ir_solve(A, b, solver=solver, tol=1e-10, inner_tol=1e-5)
    D = dense(A) if A.nrows <= 2000 else None
    res = np.linalg.norm(b - D @ r.x) / np.linalg.norm(b)
    assert r.status == 0 and res <= 1e-10
    assert r.outer >= 2  # one FP32 inner solve cannot reach 1e-10 on its own
    ref = np.linalg.solve(D, b)
    assert np.linalg.norm(r.x - ref) <= 1e-7 * np.linalg.norm(ref)


# The inexact inner stop: each FP32 inner solve runs to relative
# max(inner_tol, theta tol ||b|| / ||r_k||).  On 2D Poisson 40^2 refinement to
# 1e-10 needs three outer steps; the third starts just above the target, so
# only its inner solve may stop early.
def test_ir_theta_stops_only_the_last_inner_solve_early():
    A = W.poisson2d(40)
    b = W.vector(A.nrows, 11)
    D = dense(A)
    ref = np.linalg.solve(D, b)
    full = oracle.ir_solve(A, b, tol=1e-10, inner_tol=1e-5, theta=0.0)
    early = oracle.ir_solve(A, b, tol=1e-10, inner_tol=1e-5, theta=0.5)
    assert full.outer == early.outer == 3
    for r in (full, early):
        res = np.linalg.norm(b - D @ r.x) / np.linalg.norm(b)
        assert r.status == 0 and res <= 1e-10
        assert np.linalg.norm(r.x - ref) <= 1e-7 * np.linalg.norm(ref)
    # the third inner solve only has to take the residual from just above
    # 1e-10 ||b|| to half of that: a few steps instead of a fifth of the rest
    assert early.inner_total < full.inner_total - 50
    # the first two outer steps need reductions below inner_tol, so theta
    # leaves them alone: stopped after two, both runs hold the same iterate
    two_full = oracle.ir_solve(A, b, tol=1e-10, inner_tol=1e-5, theta=0.0, max_outer=2)
    two_early = oracle.ir_solve(A, b, tol=1e-10, inner_tol=1e-5, theta=0.5, max_outer=2)
    assert two_full.status == two_early.status == 4
    assert two_full.inner_total == two_early.inner_total
    assert np.array_equal(two_full.x, two_early.x)


@pytest.mark.parametrize("solver,make", [("cg", lambda: W.poisson2d(40)),
                                         ("gmres", lambda: W.convdiff3d(8))])
def test_ir_theta_monotone_and_scale_free(solver, make):
    A = make()
    b = W.vector(A.nrows, 11)
    runs = [oracle.ir_solve(A, b, solver=solver, tol=1e-10, theta=t) for t in (0.0, 0.5, 0.9)]
    D = dense(A)
    for r in runs:
        assert r.status == 0
        assert np.linalg.norm(b - D @ r.x) <= 1e-10 * np.linalg.norm(b)
    # a larger theta never asks an inner solve for more
    assert runs[2].inner_total <= runs[1].inner_total <= runs[0].inner_total
    # the rule is relative to ||b||: scaling b by a power of two scales every
    # FP64 and FP32 quantity exactly, so the steps and the iterate follow
    s = oracle.ir_solve(A, b * 1024.0, solver=solver, tol=1e-10, theta=0.5)
    assert (s.outer, s.inner_total) == (runs[1].outer, runs[1].inner_total)
    assert np.array_equal(s.x, runs[1].x * 1024.0)
