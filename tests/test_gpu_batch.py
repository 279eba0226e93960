"""Batched persistent solves (one launch, one block per system) vs the oracle.

Every system is checked on its own: true relative residual <= 1e-10 by the
oracle's SpMV, solution within 1e-7 of the oracle's FP64 solve; the batch's
result for a system equals its result when solved alone in a batch of one
(same kernel, same block size, same arithmetic order) to 1e-12."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_10143_b300 import cascade as C
from paper_2411_10143_b300 import workloads as W

pytestmark = pytest.mark.gpu


def systems():
    out = []
    for i, N in enumerate([6, 9, 14, 11, 5, 17]):
        out.append((W.poisson3d(N), 0))
    for N in [20, 33, 50]:
        out.append((W.poisson2d(N), 0))
    for n in [500, 3000, 9000]:
        out.append((W.spd_powerlaw(n, seed=n), 0))
    for N in [5, 9, 13, 16]:
        out.append((W.convdiff3d(N), 1))
    out.append((W.diagonally_dominant(W.powerlaw(2000, lmax=300, seed=4)), 1))
    return out


def check(ctx, sys, threads, seeds=None):
    mats = [ctx.load(A) for A, _ in sys]
    seeds = seeds if seeds is not None else list(range(len(sys)))
    rhs = [oracle.spmv(A, W.vector(A.nrows, q + 40)) for q, (A, _) in zip(seeds, sys)]
    bs = [torch.as_tensor(b, device="cuda") for b in rhs]
    xs = [torch.zeros(A.nrows, dtype=torch.float64, device="cuda") for A, _ in sys]
    infos = ctx.batch_solve(mats, [s for _, s in sys], bs, xs,
                            C.default_opts(tol=1e-10, inner_tol=1e-5, restart=30,
                                           precision=C.PREC_FP32_IR), threads)
    sols = []
    for (A, s), b, x, info in zip(sys, rhs, xs, infos):
        xh = x.cpu().numpy()
        rel = np.linalg.norm(b - oracle.spmv(A, xh)) / np.linalg.norm(b)
        ref = (oracle.cg if s == 0 else oracle.gmres)(A, b, tol=1e-10)
        assert info.status == 0 and rel <= 1e-10, (A.name, rel)
        assert np.linalg.norm(xh - ref.x) <= 1e-7 * np.linalg.norm(ref.x), A.name
        assert info.outer_iters >= 2
        sols.append(xh)
    return mats, sols


@pytest.mark.parametrize("threads", [128, 512, 0])
def test_batch_matches_oracle(threads):
    ctx = C.Context(0)
    check(ctx, systems(), threads)
    ctx.close()


def test_batch_result_same_alone_and_in_the_mix():
    ctx = C.Context(0)
    sys = systems()
    _, mixed = check(ctx, sys, 256)
    for k in (0, 7, 12):
        _, alone = check(ctx, [sys[k]], 256, seeds=[k])
        assert np.linalg.norm(alone[0] - mixed[k]) <= 1e-12 * np.linalg.norm(mixed[k])
    ctx.close()


def test_batch_rejects_bad_arguments():
    ctx = C.Context(0)
    A = W.poisson2d(8)
    M = ctx.load(A)
    b = torch.ones(64, dtype=torch.float64, device="cuda")
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(C.CascadeError):
        ctx.batch_solve([M], [2], [b], [x])
    with pytest.raises(C.CascadeError):
        ctx.batch_solve([M], [1], [b], [x], C.default_opts(restart=40, precision=1))
    with pytest.raises(C.CascadeError):
        ctx.batch_solve([M], [0], [b], [x], threads=256, threads_per_row=3)
    ctx.close()


def test_autotuner_times_every_candidate_and_its_choice_is_used():
    """cp_batch_tune times every launch shape (threads per system x threads per
    row) on a real batch (scratch solutions: the caller's x are untouched),
    records the fastest for the batch's class, and cp_batch_solve(threads=0) then
    solves with it to the same tolerance."""
    ctx = C.Context(0)
    sys = [(W.poisson2d(N), 0) for N in (40, 44, 48, 52)] + [(W.spd_powerlaw(2500, seed=9), 0)]
    mats = [ctx.load(A) for A, _ in sys]
    rhs = [oracle.spmv(A, W.vector(A.nrows, q + 70)) for q, (A, _) in enumerate(sys)]
    bs = [torch.as_tensor(b, device="cuda") for b in rhs]
    opts = C.default_opts(tol=1e-10, inner_tol=1e-5, precision=C.PREC_FP32_IR)
    best, ms, (order, ms_order) = ctx.batch_tune(mats, [s for _, s in sys], bs, opts,
                                                 with_order=True)
    assert best[0] in (128, 256, 512, 1024) and best[1] in (1, 4, 16)
    assert len(ms) == 12 and all(t > 0 for t in ms.values())
    assert ms[best] == min(ms.values())
    # the packing order: the caller's order is kept only where it timed faster
    assert ms_order > 0 and order == (1 if ms_order < ms[best] else 0)
    mean = sum(A.nrows for A, _ in sys) // len(sys)
    assert ctx.batch_schedule(mean, False) == best
    assert ctx.batch_schedule(mean, False, with_order=True) == best + (order,)
    # a class that was not tuned keeps the size rule, a thread per row
    assert ctx.batch_schedule(100, True) == (128, 1)
    assert ctx.batch_schedule(200000, True) == (1024, 1)
    assert ctx.batch_schedule(1000, True) == (256, 1) and ctx.batch_schedule(4000, True) == (512, 1)
    assert ctx.batch_schedule(4000, True, with_order=True) == (512, 1, 0)
    check(ctx, sys, 0, seeds=[q + 30 for q in range(len(sys))])
    ctx.close()


@pytest.mark.parametrize("tpv", [4, 16])
def test_batch_threads_per_row_matches_oracle(tpv):
    """Rows shared by groups of 4 or 16 lanes (shuffle sums) give the same
    solutions, on stencils, power-law rows and GMRES systems."""
    ctx = C.Context(0)
    mats = [ctx.load(A) for A, _ in systems()]
    sys = systems()
    rhs = [oracle.spmv(A, W.vector(A.nrows, q + 40)) for q, (A, _) in enumerate(sys)]
    bs = [torch.as_tensor(b, device="cuda") for b in rhs]
    xs = [torch.zeros(A.nrows, dtype=torch.float64, device="cuda") for A, _ in sys]
    infos = ctx.batch_solve(mats, [s for _, s in sys], bs, xs,
                            C.default_opts(tol=1e-10, inner_tol=1e-5, restart=30,
                                           precision=C.PREC_FP32_IR), 256, tpv)
    for (A, s), b, x, info in zip(sys, rhs, xs, infos):
        xh = x.cpu().numpy()
        rel = np.linalg.norm(b - oracle.spmv(A, xh)) / np.linalg.norm(b)
        ref = (oracle.cg if s == 0 else oracle.gmres)(A, b, tol=1e-10)
        assert info.status == 0 and rel <= 1e-10, (A.name, rel)
        assert np.linalg.norm(xh - ref.x) <= 1e-7 * np.linalg.norm(ref.x), A.name
    ctx.close()


def test_batch_inexact_inner_stop():
    """ir_theta in the batched kernel.  With inner solves to 1e-4 every system
    takes three outer steps; with theta 0.5 the third inner solve stops once it
    has brought the residual to half the target, so each system takes fewer
    inner steps.  Every system still meets the target and the oracle's
    solution, in the oracle's outer steps."""
    ctx = C.Context(0)
    sys = [(W.poisson3d(9), 0), (W.spd_powerlaw(3000, seed=3000), 0), (W.convdiff3d(9), 1),
           (W.poisson2d(33), 0)]
    mats = [ctx.load(A) for A, _ in sys]
    rhs = [oracle.spmv(A, W.vector(A.nrows, q + 40)) for q, (A, _) in enumerate(sys)]
    bs = [torch.as_tensor(b, device="cuda") for b in rhs]
    steps = {}
    for th in (0.0, 0.5):
        xs = [torch.zeros(A.nrows, dtype=torch.float64, device="cuda") for A, _ in sys]
        infos = ctx.batch_solve(mats, [s for _, s in sys], bs, xs,
                                C.default_opts(tol=1e-10, inner_tol=1e-4, restart=30,
                                               precision=C.PREC_FP32_IR, ir_theta=th), 256)
        steps[th] = [info.iters for info in infos]
        for (A, s), b, x, info in zip(sys, rhs, xs, infos):
            xh = x.cpu().numpy()
            rel = np.linalg.norm(b - oracle.spmv(A, xh)) / np.linalg.norm(b)
            ref = oracle.ir_solve(A, b, solver="cg" if s == 0 else "gmres", tol=1e-10,
                                  inner_tol=1e-4, theta=th)
            ref64 = (oracle.cg if s == 0 else oracle.gmres)(A, b, tol=1e-10)
            assert info.status == 0 and rel <= 1e-10, (A.name, th, rel)
            assert np.linalg.norm(xh - ref64.x) <= 1e-7 * np.linalg.norm(ref64.x), A.name
            assert info.outer_iters == ref.outer == 3, (A.name, th)
    assert all(a < b for a, b in zip(steps[0.5], steps[0.0])), steps
    ctx.close()


def row_length_model(ctx, threshold):
    """A BATCH_TPR classifier written by hand: class 2 (16 threads per row) when
    the longest row (feature 7, max) exceeds `threshold`, else class 0 (one
    thread per row).  With mu = 0 and sd = 1 the input is z = log(1 + f); hidden
    unit 0 is relu(z_7 - log(1 + threshold)), unit 1 relu(log(1 + threshold) -
    z_7), both passed through the second layer to the logits of classes 2 and
    0.  Returns (params, dims)."""
    d, h1, h2, k = 15, 2, 2, 3
    P = np.zeros(C.Context.mlp_nparams(d, h1, h2, k), np.float32)
    c = np.log1p(threshold)
    W1 = P[:h1 * d].reshape(h1, d)
    W1[0, 7], W1[1, 7] = 1.0, -1.0
    o = h1 * d
    P[o], P[o + 1] = -c, c  # b1
    o += h1
    W2 = P[o:o + h2 * h1].reshape(h2, h1)
    W2[0, 0] = W2[1, 1] = 1.0
    o += h2 * h1 + h2  # b2 = 0
    W3 = P[o:o + k * h2].reshape(k, h2)
    W3[2, 0] = W3[0, 1] = 1.0
    ctx.model_load(C.STAGE_BATCH_TPR, h1, h2, k, P, np.zeros(15), np.ones(15))
    return P, (d, h1, h2, k)


def test_batch_threads_per_row_per_system_from_the_classifier():
    """With a BATCH_TPR model installed, cp_batch_solve(threads_per_row = 0) gives
    each system the classifier's pick for its matrix (cp_batch_tpr: the oracle's
    forward pass on the matrix's features picks the same), so one launch mixes
    systems at 1 and at 16 threads per row.  Every system meets the oracle, and
    its result equals that of a batch of one at its own threads per row.  A new
    installation replaces the picks kept with the matrices."""
    ctx = C.Context(0)
    P, dims = row_length_model(ctx, 30)
    sys = systems()
    mats = [ctx.load(A) for A, _ in sys]
    picks = [ctx.batch_tpr(M) for M in mats]
    for (A, _), M, t in zip(sys, mats, picks):
        lg = oracle.mlp_forward(P, oracle.mlp_input(M.features(), np.zeros(15), np.ones(15)), dims)
        assert t == C.BATCH_TPR_CLASSES[int(np.argmax(lg))], A.name
        assert t == (16 if np.diff(A.rowptr).max() > 30 else 1), A.name
    assert 1 in picks and 16 in picks, picks
    _, mixed = check(ctx, sys, 256)
    for k in (0, picks.index(16), len(sys) - 1):
        bs = [torch.as_tensor(oracle.spmv(sys[k][0], W.vector(sys[k][0].nrows, k + 40)),
                              device="cuda")]
        xs = [torch.zeros(sys[k][0].nrows, dtype=torch.float64, device="cuda")]
        ctx.batch_solve([mats[k]], [sys[k][1]], bs, xs,
                        C.default_opts(tol=1e-10, inner_tol=1e-5, restart=30,
                                       precision=C.PREC_FP32_IR), 256, picks[k])
        alone = xs[0].cpu().numpy()
        assert np.linalg.norm(alone - mixed[k]) <= 1e-12 * np.linalg.norm(mixed[k]), k
    row_length_model(ctx, 1e9)  # every row is short now
    assert all(ctx.batch_tpr(M) == 1 for M in mats)
    ctx.close()


def test_batch_threads_per_row_without_a_model_is_the_schedule():
    ctx = C.Context(0)
    M = ctx.load(W.poisson2d(20))
    assert ctx.batch_tpr(M) == 0
    ctx.close()
