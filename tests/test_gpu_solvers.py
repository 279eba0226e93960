"""GPU CG / GMRES(m) / FP32-inner refinement vs the oracle, and the
asynchronous and sequential cascade modes.

Acceptance: the true relative residual of the GPU solution, recomputed by the
oracle's SpMV, is <= 1e-10, and the solution is within 1e-7 (relative) of the
oracle's own solution at the same tolerance."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_10143_b300 import cascade as C
from paper_2411_10143_b300 import workloads as W
from gpu_helpers import all_configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = C.Context(0)
    yield c
    c.close()


def true_relres(A, x, b):
    return np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)


def gpu_solve(ctx, A, b, kind="cg", x0=None, **kw):
    M = ctx.load(A)
    force = kw.pop("force", None)
    raise_on_error = kw.pop("raise_on_error", True)
    opts = C.default_opts(**kw)
    bd = torch.as_tensor(b, device="cuda")
    xd = (torch.as_tensor(x0, device="cuda").clone() if x0 is not None
          else torch.zeros(A.nrows, dtype=torch.float64, device="cuda"))
    fn = M.solve_cg if kind == "cg" else M.solve_gmres
    info = fn(bd, xd, opts, force=force, raise_on_error=raise_on_error)
    return xd.cpu().numpy(), info


def rhs(A, seed):
    return oracle.spmv(A, W.vector(A.ncols, seed))


def test_cg_poisson2d_64_plain():
    """The 2D Poisson 64x64 system (n = 4096) with the default CSR-scalar kernel."""
    c = C.Context(0)
    A = W.poisson2d(64)
    b = rhs(A, 2001)
    x, info = gpu_solve(c, A, b, tol=1e-10)
    ref = oracle.cg(A, b, tol=1e-10)
    assert info.status == 0 and true_relres(A, x, b) <= 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
    assert abs(info.iters - ref.iters) <= 3
    assert info.final_cfg.fmt == C.FMT_CSR


@pytest.mark.parametrize("ci", range(len(all_configs())))
def test_cg_every_forced_config(ctx, ci):
    cfg = all_configs()[ci]
    A = W.poisson3d(14)
    b = rhs(A, 3)
    x, info = gpu_solve(ctx, A, b, tol=1e-10, force=cfg)
    ref = oracle.cg(A, b, tol=1e-10)
    assert true_relres(A, x, b) <= 1e-10, repr(cfg)
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x), repr(cfg)


def test_cg_spd_powerlaw_and_x0(ctx):
    A = W.spd_powerlaw(20000, seed=5)
    b = rhs(A, 4)
    x0 = W.vector(A.nrows, 9)
    x, info = gpu_solve(ctx, A, b, x0=x0, tol=1e-10)
    ref = oracle.cg(A, b, tol=1e-10)
    assert true_relres(A, x, b) <= 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("m", [5, 30])
def test_gmres_convdiff(ctx, m):
    A = W.convdiff3d(12)
    b = rhs(A, 5)
    x, info = gpu_solve(ctx, A, b, kind="gmres", restart=m, tol=1e-10)
    ref = oracle.gmres(A, b, m=m, tol=1e-10)
    assert info.status == 0 and true_relres(A, x, b) <= 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("cfg", [C.config("ELL"), C.config("SELL", sigma=1024),
                                 C.config("HYB"), C.config("COO"), C.config("DIA"),
                                 C.config("CSR", C.ALGO_MERGE)])
def test_gmres_forced_configs(ctx, cfg):
    A = (W.convdiff3d(12) if cfg.fmt == C.FMT_DIA
         else W.diagonally_dominant(W.powerlaw(6000, lmax=400, seed=8)))
    b = rhs(A, 6)
    x, info = gpu_solve(ctx, A, b, kind="gmres", restart=30, tol=1e-10, force=cfg)
    ref = oracle.gmres(A, b, m=30, tol=1e-10)
    assert true_relres(A, x, b) <= 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("kind,make", [("cg", lambda: W.poisson3d(16)),
                                       ("gmres", lambda: W.convdiff3d(14)),
                                       ("cg", lambda: W.spd_powerlaw(8000, seed=2))])
def test_fp32_inner_refinement(ctx, kind, make):
    A = make()
    b = rhs(A, 7)
    x, info = gpu_solve(ctx, A, b, kind=kind, tol=1e-10, precision=C.PREC_FP32_IR,
                        inner_tol=1e-5)
    ref = oracle.ir_solve(A, b, solver=kind, tol=1e-10, inner_tol=1e-5)
    ref64 = (oracle.cg if kind == "cg" else oracle.gmres)(A, b, tol=1e-10)
    assert info.status == 0 and true_relres(A, x, b) <= 1e-10
    assert info.outer_iters >= 2
    assert np.linalg.norm(x - ref64.x) <= 1e-7 * np.linalg.norm(ref64.x)
    assert ref.status == 0


@pytest.mark.parametrize("kind,make", [("cg", lambda: W.poisson3d(16)),
                                       ("gmres", lambda: W.convdiff3d(14)),
                                       ("cg", lambda: W.spd_powerlaw(8000, seed=2))])
def test_fp32_refinement_inexact_inner_stop(ctx, kind, make):
    """ir_theta.  With inner solves to 1e-4, refinement to 1e-10 takes three
    outer steps, the second leaving a residual near 1e-8 ||b||.  The third
    inner solve then needs a reduction of about 1e-2, so with theta 0.5 it
    stops long before 1e-4.  Both settings reach the target and the FP64
    oracle's solution, in the oracle's outer steps, and theta 0.5 takes fewer
    inner steps on both sides."""
    A = make()
    b = rhs(A, 7)
    ref64 = (oracle.cg if kind == "cg" else oracle.gmres)(A, b, tol=1e-10)
    steps = {}
    for th in (0.0, 0.5):
        x, info = gpu_solve(ctx, A, b, kind=kind, tol=1e-10, precision=C.PREC_FP32_IR,
                            inner_tol=1e-4, ir_theta=th)
        ref = oracle.ir_solve(A, b, solver=kind, tol=1e-10, inner_tol=1e-4, theta=th)
        assert info.status == 0 and ref.status == 0
        assert true_relres(A, x, b) <= 1e-10
        assert np.linalg.norm(x - ref64.x) <= 1e-7 * np.linalg.norm(ref64.x)
        assert info.outer_iters == ref.outer == 3
        steps[th] = (info.iters, ref.inner_total)
    assert steps[0.5][0] < steps[0.0][0] and steps[0.5][1] < steps[0.0][1]


def test_ir_theta_out_of_range_is_rejected(ctx):
    A = W.poisson2d(10)
    for th in (-0.1, 1.0):
        with pytest.raises(C.CascadeError):
            gpu_solve(ctx, A, rhs(A, 1), precision=C.PREC_FP32_IR, ir_theta=th)


def test_edge_cases(ctx):
    A = W.poisson2d(10)
    x, info = gpu_solve(ctx, A, np.zeros(100))
    assert not x.any() and info.status == 0
    x, info = gpu_solve(ctx, A, rhs(A, 1), maxit=3, raise_on_error=False)
    assert info.status == C.ERR_NOT_CONVERGED and info.iters == 3
    neg = W.Matrix(A.nrows, A.ncols, A.rowptr, A.col, -A.val)
    x, info = gpu_solve(ctx, neg, rhs(A, 1), raise_on_error=False)
    assert info.status == C.ERR_BREAKDOWN
    x, info = gpu_solve(ctx, A, np.zeros(100), kind="gmres")
    assert not x.any() and info.status == 0


def one_hot_model(ctx, stage, cls):
    """A classifier that always answers `cls` (zero weights, one-hot output bias)."""
    k = C.STAGE_CLASSES[stage]
    n = C.Context.mlp_nparams(15, 4, 4, k)
    P = np.zeros(n, np.float32)
    P[n - k + cls] = 1.0
    ctx.model_load(stage, 4, 4, k, P, np.zeros(15), np.ones(15))


def expected_target(target):
    """(models to load, expected final configuration) for a forced cascade."""
    if target == "CSR-vector":
        return ([(C.STAGE_FORMAT, C.FMT_CSR), (C.STAGE_CSR_ALGO, C.ALGO_VECTOR),
                 (C.STAGE_CSR_TPV, 3)], ("CSR", C.ALGO_VECTOR, 16))
    return ([(C.STAGE_FORMAT, C.FORMATS.index(target)), (C.STAGE_SELL_SIGMA, 2)],
            (target, None, None))


@pytest.mark.parametrize("target", ["ELL", "SELL", "HYB", "DIA", "CSR-vector"])
def test_sequential_cascade_applies_every_stage(target):
    """SerGMRES-style: predict first, so every stage is applied at iteration 0."""
    c = C.Context(0)
    loads, (fmt, algo, tpv) = expected_target(target)
    for stage, cls in loads:
        one_hot_model(c, stage, cls)
    A = W.poisson3d(24)
    b = rhs(A, 8)
    x, info = gpu_solve(c, A, b, tol=1e-10, mode=C.MODE_SEQUENTIAL)
    ref = oracle.cg(A, b, tol=1e-10)
    assert true_relres(A, x, b) <= 1e-10
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
    assert C.FORMATS[info.final_cfg.fmt] == fmt
    if target == "CSR-vector":
        assert info.final_cfg.algo == algo and info.final_cfg.tpv == tpv
        assert info.switch_iter[0] == -1 and info.switch_iter[1] == 0 and info.switch_iter[2] == 0
    else:
        assert info.switch_iter[0] == 0
        if target == "SELL":
            assert info.final_cfg.sell_sigma == 1024
    c.close()


@pytest.mark.parametrize("target", ["ELL", "SELL", "HYB", "DIA", "CSR-vector"])
def test_async_cascade_switches_mid_run(target):
    """The solve starts at once on CSR-scalar; every prediction that lands before
    convergence is applied at a later iteration, in cascade order.  The 2D Poisson
    system on a 512^2 grid needs about two thousand CG iterations, so every stage
    lands.  The true residual is recomputed with the oracle's SpMV, and the
    solution equals the plain (never switched) solve within the solution
    tolerance."""
    c = C.Context(0)
    loads, (fmt, algo, tpv) = expected_target(target)
    for stage, cls in loads:
        one_hot_model(c, stage, cls)
    A = W.poisson2d(512)
    b = rhs(A, 8)
    x, info = gpu_solve(c, A, b, tol=1e-10, mode=C.MODE_ASYNC)
    assert true_relres(A, x, b) <= 1e-10
    xp, plain = gpu_solve(c, A, b, tol=1e-10, mode=C.MODE_PLAIN)
    assert plain.final_cfg.fmt == C.FMT_CSR and max(plain.switch_iter) == -1
    assert np.linalg.norm(x - xp) <= 1e-7 * np.linalg.norm(xp)
    applied = [s for s in info.switch_iter if s >= 0]
    assert applied == sorted(applied) and all(0 <= s <= info.iters for s in applied)
    assert C.FORMATS[info.final_cfg.fmt] == fmt
    if target == "CSR-vector":
        assert info.final_cfg.algo == algo and info.final_cfg.tpv == tpv
        assert info.switch_iter[1] >= 0 and info.switch_iter[2] >= info.switch_iter[1]
    else:
        assert info.switch_iter[0] >= 0
    assert info.t_features_ms > 0
    c.close()


def test_async_gmres_ir_switch():
    c = C.Context(0)
    one_hot_model(c, C.STAGE_FORMAT, C.FMT_SELL)
    one_hot_model(c, C.STAGE_SELL_SIGMA, 1)
    A = W.convdiff3d(20)
    b = rhs(A, 9)
    x, info = gpu_solve(c, A, b, kind="gmres", tol=1e-10, mode=C.MODE_ASYNC,
                        precision=C.PREC_FP32_IR)
    assert true_relres(A, x, b) <= 1e-10
    ref = oracle.gmres(A, b, m=30, tol=1e-10)
    assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
    assert info.final_cfg.fmt == C.FMT_SELL and info.final_cfg.sell_sigma == 32
    c.close()


def test_predict_sequential_api():
    c = C.Context(0)
    M = c.load(W.poisson2d(32))
    cfg, ms = M.predict()  # no models: CSR stays
    assert cfg.fmt == C.FMT_CSR and cfg.algo == C.ALGO_SCALAR and ms[0] > 0
    one_hot_model(c, C.STAGE_FORMAT, C.FMT_ELL)
    cfg, ms = M.predict()
    assert cfg.fmt == C.FMT_ELL
    c.close()


@pytest.mark.parametrize("cfg", [C.config("CSR"), C.config("CSR", C.ALGO_VECTOR, tpv=8),
                                 C.config("ELL"), C.config("SELL", sigma=1024), C.config("DIA"),
                                 C.config("HYB")])
@pytest.mark.parametrize("precision", [C.PREC_FP64, C.PREC_FP32_IR])
def test_persistent_cg_matches_per_step_launches(ctx, cfg, precision):
    """The persistent cooperative CG kernel and the one-launch-per-step path run the
    same iteration; both reach the tolerance and agree with the oracle."""
    A = W.poisson3d(20)
    b = rhs(A, 12)
    ref = oracle.cg(A, b, tol=1e-10)
    out = {}
    for mode in (0, 1):
        x, info = gpu_solve(ctx, A, b, tol=1e-10, force=cfg, precision=precision,
                            iteration_kernel=mode)
        assert true_relres(A, x, b) <= 1e-10, (repr(cfg), mode)
        assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
        out[mode] = (x, info)
    assert out[0][1].persist_iters > 0 and out[1][1].persist_iters == 0
    assert abs(out[0][1].iters - out[1][1].iters) <= 2


@pytest.mark.parametrize("cfg", [C.config("CSR"), C.config("CSR", C.ALGO_VECTOR, tpv=4),
                                 C.config("ELL"), C.config("SELL", sigma=32), C.config("DIA")],
                         ids=repr)
def test_two_barrier_fp32_cg_on_an_odd_order_grid(ctx, cfg):
    """The FP32 inner solves' persistent CG (two grid barriers an iteration, A p
    carried by its recurrence) on a 3D Poisson grid of odd order (n = 9261, so the
    vector loops have an odd last element), in launches of 7 iterations that
    alternate with per-step launches: every launch starts from q = A p, returns
    with p = r + beta p at its iteration limit, and the per-step path carries on
    from that state.  Against the one-launch-per-step solve and the oracle."""
    A = W.poisson3d(21)
    b = rhs(A, 15)
    ref = oracle.cg(A, b, tol=1e-10)
    runs = {}
    for mode, chunk in ((0, 0), (1, 0), (2, 7)):
        x, info = gpu_solve(ctx, A, b, tol=1e-10, force=cfg, precision=C.PREC_FP32_IR,
                            inner_tol=1e-5, iteration_kernel=mode, persist_chunk=chunk)
        assert info.status == 0 and true_relres(A, x, b) <= 1e-10, (repr(cfg), mode)
        assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
        runs[mode] = info
    assert runs[0].persist_iters > 0 and runs[1].persist_iters == 0
    assert runs[2].persist_iters > 0 and runs[2].persist_launches >= 2
    # the same iteration up to rounding: inner iteration counts within two a
    # refinement step of the per-step path's
    assert abs(runs[0].outer_iters - runs[1].outer_iters) <= 1
    assert abs(runs[0].iters - runs[1].iters) <= 2 * max(runs[0].outer_iters, 1)


@pytest.mark.parametrize("make,fmt,hyb_k", [(lambda: W.spd_powerlaw(8000, seed=2), "HYB", 0),
                                             (lambda: W.spd_powerlaw(8000, seed=2), "HYB", 2),
                                             (lambda: W.spd_powerlaw(8000, seed=2), "COO", 0),
                                             (lambda: W.poisson3d(21), "HYB", 3),
                                             (lambda: W.poisson3d(21), "COO", 0)])
@pytest.mark.parametrize("precision", [C.PREC_FP64, C.PREC_FP32_IR])
def test_persistent_cg_hyb_with_a_coo_part(ctx, make, fmt, hyb_k, precision):
    """HYB whose rows overflow the ELL width, and COO, keep the persistent CG
    kernel: the COO entries are added by lane sums, a segmented scan across
    lanes and atomics into a second buffer.  Power-law rows (runs longer than a
    warp's tile) and a 3D Poisson grid of odd order (n = 9261, an odd last
    element) against the one-launch-per-step path, the oracle, and chunked
    launches that alternate with per-step launches."""
    A = make()
    b = rhs(A, 13)
    ref = oracle.cg(A, b, tol=1e-10)
    cfg = C.config(fmt, hyb_k=hyb_k)
    runs = {}
    for mode, chunk in ((0, 0), (1, 0), (2, 7)):
        x, info = gpu_solve(ctx, A, b, tol=1e-10, force=cfg, precision=precision,
                            iteration_kernel=mode, persist_chunk=chunk)
        assert info.status == 0 and true_relres(A, x, b) <= 1e-10, (hyb_k, mode)
        assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
        assert info.final_cfg.fmt == cfg.fmt
        runs[mode] = info
    assert runs[0].persist_iters > 0 and runs[0].persist_launches >= 1
    assert runs[1].persist_iters == 0
    assert runs[2].persist_iters > 0 and runs[2].persist_launches >= 2
    assert abs(runs[0].iters - runs[1].iters) <= 2


def arrow_spd(n, seed):
    """Row 0 and column 0 dense, a diagonal elsewhere: A[0, j] = A[j, 0] = a_j
    ~ U[-1, 1], A[j, j] = 1 + |a_j|, A[0, 0] = 1 + sum |a_j| (strictly diagonally
    dominant, so SPD).  Row 0 holds n entries: in HYB's COO part and in COO it
    spans tiles of many warps and blocks, all adding into one row."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, n - 1)
    rowptr = np.zeros(n + 1, np.int32)
    rowptr[1] = n
    rowptr[2:] = n + 2 * np.arange(1, n)
    col = np.empty(n + 2 * (n - 1), np.int32)
    val = np.empty(col.size)
    col[:n] = np.arange(n)
    val[0] = 1.0 + np.abs(a).sum()
    val[1:n] = a
    col[n::2] = 0
    col[n + 1::2] = np.arange(1, n)
    val[n::2] = a
    val[n + 1::2] = 1.0 + np.abs(a)
    return W.Matrix(n, n, rowptr, col, val)


@pytest.mark.parametrize("cfg", [C.config("HYB"), C.config("COO")], ids=repr)
@pytest.mark.parametrize("kind", ["cg", "gmres"])
def test_persistent_solvers_one_dense_row(ctx, cfg, kind):
    """An arrow matrix (n = 20,001: one row of 20,001 entries) in the persistent
    kernels' COO path against the per-step launches and the oracle."""
    A = arrow_spd(20001, 5)
    b = rhs(A, 14)
    ref = oracle.cg(A, b, tol=1e-10) if kind == "cg" else oracle.gmres(A, b, m=30, tol=1e-10)
    for mode in (0, 1):
        x, info = gpu_solve(ctx, A, b, kind=kind, tol=1e-10, force=cfg, iteration_kernel=mode)
        assert info.status == 0 and true_relres(A, x, b) <= 1e-10, (kind, mode)
        assert np.linalg.norm(x - ref.x) <= 1e-7 * np.linalg.norm(ref.x)
        assert (info.persist_iters > 0) == (mode == 0)


def fixed_gate(speedup=2.0, conv_ms=5.0, spmv_ms=0.05, feat_ms=0.0, small_rows=0):
    return C.Gate.from_dict({"speedup": [1.0] + [speedup] * 5, "conv_a_ms": [0.0] + [conv_ms] * 5,
                             "conv_b_ms": [0.0] * 6, "spmv_a_ms": spmv_ms, "spmv_b_ms": 0.0,
                             "feat_a_ms": feat_ms, "feat_b_ms": 0.0, "small_rows": small_rows})


def solve_until_the_gate_decides(ctx, A, b, tries=3, **kw):
    """An asynchronous solve, repeated (up to `tries` times) until the side
    thread's gate verdict landed before the solve ended.  On a solve of a few
    milliseconds the host may schedule the side thread late enough that the
    solve converges first and no verdict is recorded (gate_remaining stays -1);
    that says nothing about the verdict, so the test looks at the first solve
    that has one."""
    for _ in range(tries):
        x, info = gpu_solve(ctx, A, b, mode=C.MODE_ASYNC, **kw)
        assert true_relres(A, x, b) <= kw.get("tol", 1e-10)
        if info.gate_remaining >= 0.0 or info.gate_declined > 0:
            break
    return x, info


def test_cost_aware_gate_keeps_the_default_on_a_short_solve():
    """A well-conditioned system converges in a few dozen iterations: with a
    conversion worth 100 default SpMVs and a 2x predicted speedup the gate keeps
    CSR-scalar (no conversion, no switch), and the solve is unaffected.  (n =
    1,048,576: the iteration count does not grow with n here, and the iterations
    are long enough that the side thread reaches the gate before the solve ends;
    at n = 262,144 the 44 iterations could end first.)"""
    c = C.Context(0)
    one_hot_model(c, C.STAGE_FORMAT, C.FMT_ELL)
    c.gate_set(fixed_gate())
    A = W.diagonally_dominant(W.poisson2d(1024), margin=0.5)  # a few dozen iterations
    b = rhs(A, 31)
    x, info = solve_until_the_gate_decides(c, A, b, tol=1e-10)
    diag = (info.gate_declined, info.gate_remaining, info.gate_cost_spmvs, info.iters)
    assert info.gate_declined == 1 and info.final_cfg.fmt == C.FMT_CSR, diag
    assert max(info.switch_iter) == -1 and info.t_convert_ms == 0.0
    assert 0.0 <= info.gate_remaining < 200.0 and info.gate_cost_spmvs == pytest.approx(100.0)
    c.close()


def test_cost_aware_gate_switches_on_a_long_solve():
    """2D Poisson on a 512^2 grid needs about two thousand CG iterations: the
    same gate converts to the predicted format and switches mid-run."""
    c = C.Context(0)
    one_hot_model(c, C.STAGE_FORMAT, C.FMT_ELL)
    c.gate_set(fixed_gate())
    A = W.poisson2d(512)
    b = rhs(A, 32)
    x, info = gpu_solve(c, A, b, tol=1e-10, mode=C.MODE_ASYNC)
    assert true_relres(A, x, b) <= 1e-10
    assert info.gate_declined == 0 and info.final_cfg.fmt == C.FMT_ELL
    assert info.switch_iter[0] >= 0 and info.gate_remaining > 200.0
    c.close()


def test_gate_switches_at_once_when_the_conversion_pays_back_within_a_few_iterations():
    """A 16x format whose conversion costs 2.5 default SpMVs pays back within 2.7
    iterations (cp_gate_payback): the side thread converts without waiting for
    residual history, so the gate makes no estimate of the iterations left (-1)
    and the solve switches mid-run."""
    c = C.Context(0)
    one_hot_model(c, C.STAGE_FORMAT, C.FMT_ELL)
    g = fixed_gate(speedup=16.0, conv_ms=0.125)
    assert C.gate_payback(g, C.FMT_ELL, 10**6) == pytest.approx(2.5 / (1 - 1 / 16))
    c.gate_set(g)
    A = W.poisson2d(512)
    b = rhs(A, 33)
    x, info = gpu_solve(c, A, b, tol=1e-10, mode=C.MODE_ASYNC)
    assert true_relres(A, x, b) <= 1e-10
    assert info.gate_declined == 0 and info.final_cfg.fmt == C.FMT_ELL
    assert info.switch_iter[0] >= 0
    assert info.gate_remaining == -1.0 and info.gate_cost_spmvs == pytest.approx(2.5)
    c.close()


def test_gate_neighbours_decide_with_the_matrix_own_speedup():
    """With neighbours installed the gate takes the predicted format's speedup
    from the training matrices nearest to this one.  The long solve above
    switches on the global 2x; told by its neighbours that ELL gains 1 %, the
    gate keeps CSR-scalar (about 2,000 iterations x 0.01 is below the 100-SpMV
    conversion); told 3x, it switches; with the neighbours removed, the global
    figure applies again."""
    c = C.Context(0)
    one_hot_model(c, C.STAGE_FORMAT, C.FMT_ELL)
    c.gate_set(fixed_gate())
    A = W.poisson2d(512)
    b = rhs(A, 32)
    z = np.random.default_rng(3).standard_normal((9, 15)).astype(np.float32)
    mu, sd = np.zeros(15), np.ones(15)
    for s_ell, keeps in ((1.01, True), (3.0, False)):
        sp = np.ones((9, 6), np.float32)
        sp[:, C.FMT_ELL] = s_ell
        c.gate_set_neighbours(z, sp, mu, sd, k=5)
        x, info = gpu_solve(c, A, b, tol=1e-10, mode=C.MODE_ASYNC)
        assert true_relres(A, x, b) <= 1e-10
        diag = (s_ell, info.gate_declined, info.gate_remaining, info.gate_cost_spmvs)
        if keeps:
            assert info.gate_declined == 1 and info.final_cfg.fmt == C.FMT_CSR, diag
        else:
            assert info.gate_declined == 0 and info.final_cfg.fmt == C.FMT_ELL, diag
    c.gate_set_neighbours(None)
    x, info = gpu_solve(c, A, b, tol=1e-10, mode=C.MODE_ASYNC)
    assert info.gate_declined == 0 and info.final_cfg.fmt == C.FMT_ELL
    c.close()


def test_shipped_gate_keeps_csr_where_the_predicted_format_barely_gains():
    """The shipped cascade picks SELL for 3D Poisson 48^3 (n 110,592), whose SpMV
    is about 1.05x CSR-scalar's there: over the 100-odd iterations left that
    saves less than the conversion costs, and the gate, with the shipped
    neighbours, keeps CSR-scalar."""
    from paper_2411_10143_b300 import models
    c = C.Context(0)
    assert "GATE_NEIGHBOURS" in models.load_default(c)
    A = W.poisson3d(48)
    b = rhs(A, 34)
    x, info = solve_until_the_gate_decides(c, A, b, tol=1e-10)
    diag = (info.gate_declined, info.gate_remaining, info.gate_cost_spmvs, repr(info.final_cfg))
    assert info.gate_declined == 1 and info.final_cfg.fmt == C.FMT_CSR, diag
    c.close()


def test_two_tier_features_skip_the_feature_pass_on_a_short_small_solve():
    """Below small_rows rows the side thread first asks whether even the best
    format could pay for the O(nnz) feature pass plus a conversion; on a
    well-conditioned small system it cannot, so no feature is computed and the
    solve stays on CSR-scalar."""
    c = C.Context(0)
    one_hot_model(c, C.STAGE_FORMAT, C.FMT_ELL)
    c.gate_set(fixed_gate(feat_ms=20.0, small_rows=100_000))
    # n 90,000: about 120 iterations, far fewer than the 500 SpMVs the features and
    # a conversion cost, yet long enough (a few ms) that the side thread's verdict
    # usually lands before the solve ends
    A = W.diagonally_dominant(W.poisson2d(300), margin=0.05)
    b = rhs(A, 33)
    x, info = solve_until_the_gate_decides(c, A, b, tol=1e-10)
    diag = (info.gate_declined, info.gate_remaining, info.gate_cost_spmvs, info.iters)
    assert info.gate_declined == 2 and info.t_features_ms == 0.0, diag
    assert info.final_cfg.fmt == C.FMT_CSR and max(info.switch_iter) == -1
    assert info.gate_cost_spmvs == pytest.approx((20.0 + 5.0) / 0.05)
    c.close()


def test_bounded_device_wait_times_out_cleanly():
    """The persistent kernel's grid barrier gives up after wait_limit_ms.  With a
    limit of one nanosecond its first wait runs out: every block leaves at its
    next barrier, the solve ends with CP_ERR_TIMEOUT (no fault, no hang), and the
    same context then solves normally."""
    c = C.Context(0)
    A = W.poisson3d(24)
    b = rhs(A, 44)
    x, info = gpu_solve(c, A, b, tol=1e-10, force=C.config("DIA"), raise_on_error=False,
                        wait_limit_ms=1e-6)
    assert info.status == C.ERR_TIMEOUT and info.persist_iters == 0
    x, info = gpu_solve(c, A, b, tol=1e-10, force=C.config("DIA"))
    assert info.status == 0 and true_relres(A, x, b) <= 1e-10
    c.close()


@pytest.mark.parametrize("point", [0, 1, 2])
def test_prediction_side_failure_leaves_the_solve_on_the_default_kernel(point):
    """Fault injected on the host: the side thread fails before the feature pass,
    after it, or after the FORMAT stage.  The asynchronous solve carries on with
    CSR-scalar, converges, and reports the side's error."""
    c = C.Context(0)
    one_hot_model(c, C.STAGE_FORMAT, C.FMT_ELL)
    A = W.poisson2d(256)
    b = rhs(A, 45 + point)
    c.inject_side_failure(point)
    x, info = gpu_solve(c, A, b, tol=1e-10, mode=C.MODE_ASYNC)
    assert info.status == 0 and true_relres(A, x, b) <= 1e-10
    assert info.side_status == C.ERR_CUDA
    assert info.final_cfg.fmt == C.FMT_CSR and max(info.switch_iter) == -1
    # one-shot: the next solve predicts and switches as usual
    x, info = gpu_solve(c, A, b, tol=1e-10, mode=C.MODE_ASYNC)
    assert info.side_status == 0 and info.final_cfg.fmt == C.FMT_ELL
    c.close()


def test_warmup_makes_the_first_solve_as_fast_as_the_next():
    """cp_warmup launches every solve-path kernel once on its own small system
    (with and without installed models).  After it, the process's first
    asynchronous GMRES(30) solve of a mid-size system takes about what the
    second does: no kernel's first-launch cost lands inside a solve."""
    import time
    from paper_2411_10143_b300 import models
    bare = C.Context(0)
    bare.warmup()  # no models installed: the cascade's inference is skipped
    bare.close()
    c = C.Context(0)
    models.load_default(c)
    t0 = time.perf_counter()
    c.warmup()
    assert time.perf_counter() - t0 < 10.0
    A = W.convdiff3d(48)
    b = rhs(A, 46)
    M = c.load(A)
    bd = torch.as_tensor(b, device="cuda")
    times = []
    for _ in range(2):
        M.reset()
        xd = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(c.stream)
        info = M.solve_gmres(bd, xd, C.default_opts(tol=1e-10, restart=30, mode=C.MODE_ASYNC))
        e1.record(c.stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        assert info.status == 0 and true_relres(A, xd.cpu().numpy(), b) <= 1e-10
    assert times[0] <= 1.5 * times[1] + 3.0, times
    c.close()
