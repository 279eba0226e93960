"""The persistent GMRES(m) kernel (one cooperative launch across Arnoldi steps,
cycle ends and restarts) against the one-launch-per-step path and the oracle.

Acceptance as for every solver test: the true relative residual of the GPU
solution, recomputed by the oracle's SpMV, is <= 1e-10 and the solution is
within 1e-7 (relative) of the oracle's GMRES(m) solution at the same
tolerance.  The persistent kernel orthogonalises with modified Gram-Schmidt
(in groups of four columns, one grid reduction per group) unless gmres_orth = 1
asks for classical Gram-Schmidt with a second pass, which is also what the
per-step launches and the persistent kernel on systems too large for the
shared-memory path use; iteration counts may differ by a few between them."""
import functools

import numpy as np
import pytest
import torch

import oracle
from paper_2411_10143_b300 import cascade as C
from paper_2411_10143_b300 import workloads as W

pytestmark = pytest.mark.gpu

# Configurations the persistent kernel runs.  SELL with sigma > 1 permutes rows
# inside its sorting windows, so its SpMV rows are not the block's own rows and
# the kernel takes a grid barrier after the SpMV.  HYB with K = 3 has a COO part
# on the 7-point stencil, and COO is all COO part: their COO entries go through
# atomics into a zeroed vector, a grid barrier, then each block's own rows.
CFGS = [C.config("CSR"), C.config("CSR", C.ALGO_VECTOR, tpv=4),
        C.config("CSR", C.ALGO_VECTOR, tpv=32), C.config("ELL"), C.config("SELL", sigma=1),
        C.config("SELL", sigma=1024), C.config("DIA"), C.config("HYB"),
        C.config("HYB", hyb_k=3), C.config("COO")]


@pytest.fixture(scope="module")
def ctx():
    c = C.Context(0)
    yield c
    c.close()


def true_relres(A, x, b):
    return np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)


def solve(ctx, A, b, **kw):
    M = ctx.load(A)
    force = kw.pop("force", None)
    raise_on_error = kw.pop("raise_on_error", True)
    bd = torch.as_tensor(b, device="cuda")
    xd = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    info = M.solve_gmres(bd, xd, C.default_opts(**kw), force=force,
                         raise_on_error=raise_on_error)
    return xd.cpu().numpy(), info


@functools.lru_cache(maxsize=None)
def system(k, seed):
    """Convection-diffusion on a k^3 grid with b = A x*, and the oracle's
    GMRES(m) solutions by m."""
    A = W.convdiff3d(k)
    b = oracle.spmv(A, W.vector(A.ncols, seed))
    return A, b


@functools.lru_cache(maxsize=None)
def reference(k, seed, m):
    A, b = system(k, seed)
    return oracle.gmres(A, b, m=m, tol=1e-10)


def check(A, b, x, ref):
    assert true_relres(A, x, b) <= 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)


def close_iters(a, b):
    return abs(a - b) <= max(3, 0.05 * b)


@pytest.mark.parametrize("cfg", CFGS, ids=repr)
@pytest.mark.parametrize("m", [5, 30])
def test_persistent_gmres_matches_per_step_launches(ctx, cfg, m):
    """n = 2,744: three of the 148 blocks own rows (the last one a ragged
    segment), the others none; m = 5 restarts inside the kernel many times."""
    A, b = system(14, 21)
    ref = reference(14, 21, m)
    out = {}
    for kernel in (0, 1):
        x, info = solve(ctx, A, b, restart=m, tol=1e-10, force=cfg, iteration_kernel=kernel)
        assert info.status == 0, (repr(cfg), kernel)
        check(A, b, x, ref)
        out[kernel] = info
    assert out[0].persist_iters == out[0].iters and out[0].persist_launches >= 1
    assert out[1].persist_iters == 0 and out[1].persist_launches == 0
    assert close_iters(out[0].iters, out[1].iters), (out[0].iters, out[1].iters)


@pytest.mark.parametrize("cfg", [C.config("CSR"), C.config("CSR", C.ALGO_VECTOR, tpv=4),
                                 C.config("SELL", sigma=1024), C.config("DIA"),
                                 C.config("HYB", hyb_k=3), C.config("COO")], ids=repr)
@pytest.mark.parametrize("precision", [C.PREC_FP64, C.PREC_FP32_IR])
@pytest.mark.parametrize("m", [4, 30])
def test_persistent_gmres_classical_orthogonalisation(ctx, cfg, precision, m):
    """gmres_orth = 1: the persistent kernel's classical Gram-Schmidt with the
    second pass (the path of systems whose rows do not fit in shared memory)."""
    A, b = system(14, 31)
    ref = reference(14, 31, m)
    x, info = solve(ctx, A, b, restart=m, tol=1e-10, force=cfg, gmres_orth=1,
                    precision=precision, inner_tol=1e-5)
    assert info.status == 0 and info.persist_iters == info.iters
    check(A, b, x, ref)


@pytest.mark.parametrize("cfg", [C.config("DIA"), C.config("CSR", C.ALGO_VECTOR, tpv=4),
                                 C.config("SELL", sigma=1024), C.config("HYB", hyb_k=3),
                                 C.config("COO")], ids=repr)
def test_persistent_gmres_rows_in_several_segments(ctx, cfg):
    """n = 175,616 is more than one row per thread of the grid, so every block
    owns several row segments (CSR-vector with 4 lanes a row: segments of 256
    rows)."""
    A, b = system(56, 22)
    ref = reference(56, 22, 30)
    x, info = solve(ctx, A, b, restart=30, tol=1e-10, force=cfg)
    assert info.status == 0 and info.persist_iters == info.iters
    check(A, b, x, ref)
    assert close_iters(info.iters, ref.iters), (info.iters, ref.iters)


@functools.lru_cache(maxsize=None)
def powerlaw_system():
    """A diagonally dominant nonsymmetric power-law matrix (n = 6,000, rows up to
    400 entries) with b = A x*, and the oracle's GMRES(30) solution."""
    A = W.diagonally_dominant(W.powerlaw(6000, lmax=400, seed=8))
    b = oracle.spmv(A, W.vector(A.ncols, 23))
    return A, b, oracle.gmres(A, b, m=30, tol=1e-10)


@pytest.mark.parametrize("cfg", [C.config("HYB"), C.config("HYB", hyb_k=1), C.config("COO")],
                         ids=repr)
@pytest.mark.parametrize("precision", [C.PREC_FP64, C.PREC_FP32_IR])
def test_persistent_gmres_power_law_coo_entries(ctx, cfg, precision):
    """Power-law rows (COO runs of several hundred entries across lanes, warps
    and blocks) through the persistent kernel's atomic COO path, in both
    precisions, against the per-step launches and the oracle."""
    A, b, ref = powerlaw_system()
    out = {}
    for kernel in (0, 1):
        x, info = solve(ctx, A, b, restart=30, tol=1e-10, force=cfg, iteration_kernel=kernel,
                        precision=precision, inner_tol=1e-5)
        assert info.status == 0, (repr(cfg), kernel)
        check(A, b, x, ref)
        out[kernel] = info
    assert out[0].persist_iters == out[0].iters and out[0].persist_launches >= 1
    assert out[1].persist_iters == 0


@pytest.mark.parametrize("m", [1, 3, 4, 8, 9, 17])
@pytest.mark.parametrize("precision", [C.PREC_FP64, C.PREC_FP32_IR])
def test_persistent_gmres_short_restarts(ctx, m, precision):
    """Restart lengths around the column groups the kernel's modified
    Gram-Schmidt handles per grid reduction (four in FP64, eight in FP32): one
    column (GMRES(1)), partial groups, exactly one or two groups, and full groups
    followed by a one-column group."""
    A, b = system(10, 30)
    ref = reference(10, 30, m)
    x, info = solve(ctx, A, b, restart=m, tol=1e-10, force=C.config("DIA"), maxit=20000,
                    precision=precision, inner_tol=1e-5)
    assert info.status == 0 and info.persist_iters == info.iters
    check(A, b, x, ref)
    if precision == C.PREC_FP64:
        assert close_iters(info.iters, ref.iters), (info.iters, ref.iters)


@pytest.mark.parametrize("cfg", [C.config("DIA"), C.config("CSR")], ids=repr)
def test_persistent_gmres_largest_restart(ctx, cfg):
    """m = 64, the largest restart: the kernel's shared memory (the cycle's
    Hessenberg matrix in every block) exceeds the 48 KB default and is opted in."""
    A, b = system(14, 23)
    ref = reference(14, 23, 64)
    x, info = solve(ctx, A, b, restart=64, tol=1e-10, force=cfg)
    assert info.status == 0 and info.persist_iters == info.iters
    check(A, b, x, ref)


def test_persistent_gmres_tiny_system(ctx):
    """n = 27: one block owns every row, one warp has the only chunk of dot work."""
    A, b = system(3, 24)
    ref = reference(3, 24, 30)
    x, info = solve(ctx, A, b, restart=30, tol=1e-10, force=C.config("CSR"))
    assert info.status == 0
    check(A, b, x, ref)


@pytest.mark.parametrize("cfg", [C.config("DIA"), C.config("CSR"),
                                 C.config("SELL", sigma=1024)], ids=repr)
def test_persistent_gmres_fp32_inner_solves(ctx, cfg):
    """FP64 refinement around FP32 GMRES(30) inner solves, every inner step in
    the persistent kernel."""
    A, b = system(20, 25)
    ref64 = reference(20, 25, 30)
    out = {}
    for kernel in (0, 1):
        x, info = solve(ctx, A, b, restart=30, tol=1e-10, force=cfg, iteration_kernel=kernel,
                        precision=C.PREC_FP32_IR, inner_tol=1e-5)
        assert info.status == 0 and info.outer_iters >= 2
        check(A, b, x, ref64)
        out[kernel] = info
    assert out[0].persist_iters == out[0].iters and out[1].persist_iters == 0


@pytest.mark.parametrize("chunk", [1, 7])
def test_persistent_gmres_returns_and_resumes(ctx, chunk):
    """persist_chunk makes every launch return after `chunk` steps: with m = 5
    and 7 steps a launch it returns inside cycles (columns normalised, the state
    handed back) and at their ends (x updated); the next launch resumes there.
    The solution is the same as with one launch."""
    A, b = system(14, 26)
    ref = reference(14, 26, 5)
    x1, one = solve(ctx, A, b, restart=5, tol=1e-10, force=C.config("DIA"))
    x, info = solve(ctx, A, b, restart=5, tol=1e-10, force=C.config("DIA"),
                    persist_chunk=chunk)
    assert info.status == 0 and one.persist_launches == 1
    assert info.persist_iters == info.iters
    assert info.persist_launches >= info.iters // chunk
    check(A, b, x, ref)
    assert close_iters(info.iters, one.iters)


def test_persistent_cg_returns_and_resumes(ctx):
    A = W.poisson3d(20)
    b = oracle.spmv(A, W.vector(A.ncols, 27))
    ref = oracle.cg(A, b, tol=1e-10)
    M = ctx.load(A)
    bd = torch.as_tensor(b, device="cuda")
    xd = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    info = M.solve_cg(bd, xd, C.default_opts(tol=1e-10, persist_chunk=10),
                      force=C.config("DIA"))
    x = xd.cpu().numpy()
    assert info.status == 0 and info.persist_launches >= info.iters // 10
    assert true_relres(A, x, b) <= 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)


def test_persistent_gmres_iteration_budget(ctx):
    """maxit = 13 with m = 5: the kernel ends the third cycle after 3 steps and
    returns; the solve reports CP_ERR_NOT_CONVERGED after exactly 13 steps."""
    A, b = system(14, 28)
    x, info = solve(ctx, A, b, restart=5, tol=1e-10, maxit=13, force=C.config("DIA"),
                    raise_on_error=False)
    assert info.status == C.ERR_NOT_CONVERGED and info.iters == 13
    assert info.persist_iters == 13


def test_persistent_gmres_bounded_wait_times_out_cleanly():
    """A barrier wait limit of one nanosecond: the first grid barrier gives up,
    every block leaves at its next barrier, the solve returns CP_ERR_TIMEOUT, and
    the context then solves normally."""
    c = C.Context(0)
    A, b = system(14, 29)
    x, info = solve(c, A, b, restart=30, tol=1e-10, force=C.config("DIA"),
                    raise_on_error=False, wait_limit_ms=1e-6)
    assert info.status == C.ERR_TIMEOUT
    x, info = solve(c, A, b, restart=30, tol=1e-10, force=C.config("DIA"))
    assert info.status == 0 and true_relres(A, x, b) <= 1e-10
    c.close()


@pytest.mark.parametrize("m,chunk", [(30, 7), (5, 3)])
@pytest.mark.parametrize("precision", [C.PREC_FP64, C.PREC_FP32_IR])
def test_gmres_hand_over_between_persistent_and_per_step(ctx, m, chunk, precision):
    """iteration_kernel = 2 alternates persistent launches of `chunk` steps with
    as many one-launch-per-step steps, inside cycles and across their ends: the
    persistent kernel normalises its columns and hands the cycle's state back,
    the per-step kernels extend the cycle with classical Gram-Schmidt, and the
    persistent kernel takes the cycle up again (its group inner products of the
    per-step columns being zero).  The solution is the oracle's."""
    A, b = system(14, 32)
    ref = reference(14, 32, m)
    x, info = solve(ctx, A, b, restart=m, tol=1e-10, force=C.config("DIA"), iteration_kernel=2,
                    persist_chunk=chunk, precision=precision, inner_tol=1e-5)
    assert info.status == 0
    assert 0 < info.persist_iters < info.iters and info.persist_launches >= 2
    check(A, b, x, ref)


@pytest.mark.parametrize("precision", [C.PREC_FP64, C.PREC_FP32_IR])
def test_cg_hand_over_between_persistent_and_per_step(ctx, precision):
    A = W.poisson3d(20)
    b = oracle.spmv(A, W.vector(A.ncols, 33))
    ref = oracle.cg(A, b, tol=1e-10)
    M = ctx.load(A)
    bd = torch.as_tensor(b, device="cuda")
    xd = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
    info = M.solve_cg(bd, xd, C.default_opts(tol=1e-10, iteration_kernel=2, persist_chunk=9,
                                             precision=precision, inner_tol=1e-5),
                      force=C.config("DIA"))
    x = xd.cpu().numpy()
    assert info.status == 0 and 0 < info.persist_iters < info.iters
    assert info.persist_launches >= 2
    assert true_relres(A, x, b) <= 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)


def test_alternating_mode_needs_a_chunk(ctx):
    A, b = system(3, 34)
    with pytest.raises(Exception):
        solve(ctx, A, b, iteration_kernel=2, persist_chunk=0)
