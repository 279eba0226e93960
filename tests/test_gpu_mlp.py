"""GPU predictor kernels (forward, loss + gradient, Adam) vs the FP64 oracle,
and GPU training of a cascade stage.  The GPU computes in FP32: outputs and
gradients must agree with the FP64 oracle to 1e-4 relative (norm-wise)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_10143_b300 import cascade as C

pytestmark = pytest.mark.gpu
DIMS = (15, 32, 16, 5)


@pytest.fixture(scope="module")
def ctx():
    c = C.Context(0)
    yield c
    c.close()


def setup(N, seed):
    rng = np.random.default_rng(seed)
    P = rng.normal(0, 0.4, C.Context.mlp_nparams(*DIMS)).astype(np.float32)
    X = rng.normal(size=(N, 15)).astype(np.float32)
    lab = rng.integers(0, DIMS[3], N).astype(np.int32)
    return P, X, lab


def dev(a):
    return torch.as_tensor(a, device="cuda")


@pytest.mark.parametrize("N", [1, 7, 300])
def test_forward_and_gradient_vs_oracle(ctx, N):
    P, X, lab = setup(N, N)
    scratch = torch.zeros(C.Context.mlp_scratch_floats(N, *DIMS), device="cuda")
    logits = torch.zeros((N, DIMS[3]), device="cuda")
    ctx.mlp_forward(DIMS, dev(P), dev(X), logits, scratch)
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(len(P), device="cuda")
    ctx.mlp_loss_grad(DIMS, dev(P), dev(X), dev(lab), loss, grad, scratch)
    torch.cuda.synchronize()
    ref_logits = oracle.mlp_forward(P.astype(np.float64), X.astype(np.float64), DIMS)
    ref_loss, ref_grad = oracle.mlp_loss_grad(P.astype(np.float64), X.astype(np.float64), lab, DIMS)
    lg = logits.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(lg - ref_logits) <= 1e-4 * np.linalg.norm(ref_logits)
    assert loss.item() == pytest.approx(ref_loss, rel=1e-4)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref_grad) <= 1e-4 * np.linalg.norm(ref_grad)


def test_adam_vs_oracle(ctx):
    rng = np.random.default_rng(1)
    n = 500
    P = rng.normal(size=n)
    G = rng.normal(size=n)
    m = rng.normal(size=n) * 0.1
    v = np.abs(rng.normal(size=n)) * 0.01
    Pd, Gd, md, vd = (dev(a.astype(np.float32)) for a in (P, G, m, v))
    ctx.adam_step(Pd, Gd, md, vd, 3, lr=0.01)
    torch.cuda.synchronize()
    oracle.adam_step(P, G, m, v, 3, lr=0.01)
    for a, b in ((Pd, P), (md, m), (vd, v)):
        assert np.allclose(a.cpu().numpy(), b, rtol=1e-5, atol=1e-6)


def test_train_stage_learns_separable_labels(ctx):
    rng = np.random.default_rng(5)
    N = 600
    F = np.exp(rng.uniform(0, 12, size=(N, 15)))
    # the format label depends on two features (nnz and max)
    lab = ((np.log(F[:, 2]) > 6).astype(int) + 2 * (np.log(F[:, 7]) > 6).astype(int)).astype(np.int32)
    loss = ctx.model_train(C.STAGE_FORMAT, F, lab, h1=32, h2=32, epochs=1500, lr=3e-3, seed=3)
    assert loss < 0.15
    m = ctx.model_get(C.STAGE_FORMAT)
    z = oracle.mlp_input(F, m["mu"].astype(np.float64), m["sd"].astype(np.float64))
    pred = oracle.mlp_forward(m["params"].astype(np.float64), z, m["dims"]).argmax(1)
    assert (pred == lab).mean() > 0.95


@pytest.mark.parametrize("N", [1, 7, 300])
def test_soft_target_loss_and_gradient_vs_oracle(ctx, N):
    """Cross-entropy against target distributions (the cascade's training on
    measured times): loss and gradient against the FP64 oracle, 1e-4."""
    P, X, _ = setup(N, N + 50)
    rng = np.random.default_rng(N)
    Q = rng.random((N, DIMS[3])) ** 3
    Q = (Q / Q.sum(axis=1, keepdims=True)).astype(np.float32)
    scratch = torch.zeros(C.Context.mlp_scratch_floats(N, *DIMS), device="cuda")
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(len(P), device="cuda")
    ctx.mlp_loss_grad_soft(DIMS, dev(P), dev(X), dev(Q), loss, grad, scratch)
    torch.cuda.synchronize()
    ref_loss, ref_grad = oracle.mlp_loss_grad_soft(P.astype(np.float64), X.astype(np.float64),
                                                   Q.astype(np.float64), DIMS)
    assert loss.item() == pytest.approx(ref_loss, rel=1e-4)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - ref_grad) <= 1e-4 * np.linalg.norm(ref_grad)


def test_train_stage_on_soft_targets(ctx):
    """Soft targets concentrated on the separable label train as the labels do;
    rows that are not distributions are rejected."""
    rng = np.random.default_rng(6)
    N = 600
    F = np.exp(rng.uniform(0, 12, size=(N, 15)))
    lab = ((np.log(F[:, 2]) > 6).astype(int) + 2 * (np.log(F[:, 7]) > 6).astype(int))
    Q = np.full((N, 6), 0.02)
    Q[np.arange(N), lab] = 0.9
    ctx.model_train_soft(C.STAGE_FORMAT, F, Q, h1=32, h2=32, epochs=1500, lr=3e-3, seed=3)
    m = ctx.model_get(C.STAGE_FORMAT)
    z = oracle.mlp_input(F, m["mu"].astype(np.float64), m["sd"].astype(np.float64))
    pred = oracle.mlp_forward(m["params"].astype(np.float64), z, m["dims"]).argmax(1)
    assert (pred == lab).mean() > 0.95
    with pytest.raises(C.CascadeError) as e:
        ctx.model_train_soft(C.STAGE_FORMAT, F[:4], np.full((4, 6), 0.5), epochs=1)
    assert e.value.status == C.ERR_INVALID
