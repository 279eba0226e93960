"""Pins of the oracle's predictor MLP: finite differences, an independent NumPy forward
pass, the uniform-logit loss and the closed form of Adam's first step."""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle

DIMS = (15, 8, 6, 5)
GOLDEN = Path(__file__).resolve().parent / "golden"


def params(seed, dims=DIMS, scale=0.5):
    return np.random.default_rng(seed).normal(0, scale, oracle.mlp_nparams(*dims))


def unpack(P, dims):
    d, h1, h2, k = dims
    o = 0
    out = []
    for shape in [(h1, d), (h1,), (h2, h1), (h2,), (k, h2), (k,)]:
        size = int(np.prod(shape))
        out.append(P[o:o + size].reshape(shape))
        o += size
    return out


def test_forward_matches_numpy_matrix_form():
    P = params(1)
    X = np.random.default_rng(2).normal(size=(9, 15))
    W1, b1, W2, b2, W3, b3 = unpack(P, DIMS)
    ref = np.maximum(np.maximum(X @ W1.T + b1, 0) @ W2.T + b2, 0) @ W3.T + b3
    assert np.allclose(oracle.mlp_forward(P, X, DIMS), ref, rtol=1e-13, atol=1e-13)


def test_loss_uniform_logits_is_log_k():
    P = np.zeros(oracle.mlp_nparams(*DIMS))
    X = np.random.default_rng(0).normal(size=(4, 15))
    loss, g = oracle.mlp_loss_grad(P, X, [0, 1, 2, 3], DIMS)
    assert loss == pytest.approx(math.log(5), rel=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_central_differences(seed):
    P = params(seed)
    rng = np.random.default_rng(seed + 10)
    X = rng.normal(size=(6, 15))
    lab = rng.integers(0, 5, 6)
    _, g = oracle.mlp_loss_grad(P, X, lab, DIMS)
    h = 1e-6
    num = np.empty_like(P)
    for i in range(len(P)):
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        num[i] = (oracle.mlp_loss_grad(Pp, X, lab, DIMS)[0]
                  - oracle.mlp_loss_grad(Pm, X, lab, DIMS)[0]) / (2 * h)
    # ReLU kinks are measure-zero for random inputs; central differences are O(h^2)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_adam_first_step_closed_form():
    """With m = v = 0 and t = 1 the bias corrections give P -= lr * g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    P = rng.normal(size=50)
    G = rng.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    P0 = P.copy()
    oracle.adam_step(P, G, m, v, 1, lr=0.01, eps=1e-8)
    assert np.allclose(P, P0 - 0.01 * G / (np.abs(G) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.allclose(m, 0.1 * G) and np.allclose(v, 0.001 * G * G)


def test_training_decreases_loss():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(64, 15))
    lab = (X[:, 0] > 0).astype(int) + 2 * (X[:, 1] > 0).astype(int)
    P = params(5, scale=0.3)
    m = np.zeros_like(P)
    v = np.zeros_like(P)
    l0 = oracle.mlp_loss_grad(P, X, lab, DIMS)[0]
    for t in range(1, 301):
        loss, g = oracle.mlp_loss_grad(P, X, lab, DIMS)
        oracle.adam_step(P, g, m, v, t, lr=0.01)
    assert loss < 0.3 * l0


def test_cascade_control_flow():
    # CSR -> algorithm stage -> vector -> TpV stage
    assert oracle.cascade([5, 0, 0, 0, 0], [0, 9, 0], [0, 0, 7, 0, 0]) == (0, 1, 2)
    # CSR scalar: no TpV stage
    assert oracle.cascade([5, 0, 0, 0, 0], [9, 0, 0], [0, 0, 7, 0, 0]) == (0, 0, -1)
    # SELL: sigma stage
    assert oracle.cascade([0, 0, 0, 5, 0], [9, 0, 0], None, [0, 3, 0, 0]) == (3, -1, 1)
    # ELL: nothing further
    assert oracle.cascade([0, 0, 5, 0, 0], [9, 0, 0], [1, 0, 0, 0, 0], [1, 0, 0, 0]) == (2, -1, -1)


def test_mlp_input_worked_example():
    """Hand-derived fixture: log(1 + f) is an exact multiple of log 2, log 3 or
    log 10 and mu, sd are short binary fractions, so every z is a closed form.
    A log in place of log1p, swapped mu and sd, or a sign error fails it."""
    g = json.loads((GOLDEN / "mlp_input_worked.json").read_text())
    z = oracle.mlp_input(g["f"], g["mu"], g["sd"])
    assert np.allclose(z, g["z"], rtol=2e-15, atol=2e-15), z - np.asarray(g["z"])


def test_mlp_input_is_increasing_in_each_feature():
    """The input map is strictly increasing in f_j (sd > 0): a larger feature can
    never give a smaller classifier input."""
    rng = np.random.default_rng(6)
    mu, sd = rng.normal(size=15), rng.uniform(0.1, 3, 15)
    f = rng.uniform(0, 1e6, (50, 15))
    f.sort(axis=0)
    z = np.stack([oracle.mlp_input(r, mu, sd) for r in f])
    assert np.all(np.diff(z, axis=0) >= 0)


def soft_targets(n, k, seed):
    rng = np.random.default_rng(seed)
    Q = rng.random((n, k)) ** 3
    return Q / Q.sum(axis=1, keepdims=True)


@pytest.mark.parametrize("seed", [0, 1])
def test_soft_gradient_central_differences(seed):
    P = params(seed)
    rng = np.random.default_rng(seed + 20)
    X = rng.normal(size=(6, 15))
    Q = soft_targets(6, DIMS[3], seed)
    _, g = oracle.mlp_loss_grad_soft(P, X, Q, DIMS)
    h = 1e-6
    num = np.empty_like(P)
    for i in range(len(P)):
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        num[i] = (oracle.mlp_loss_grad_soft(Pp, X, Q, DIMS)[0]
                  - oracle.mlp_loss_grad_soft(Pm, X, Q, DIMS)[0]) / (2 * h)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_soft_targets_one_hot_reduce_to_labels():
    P = params(3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(9, 15))
    lab = rng.integers(0, DIMS[3], 9)
    Q = np.eye(DIMS[3])[lab]
    l1, g1 = oracle.mlp_loss_grad(P, X, lab, DIMS)
    l2, g2 = oracle.mlp_loss_grad_soft(P, X, Q, DIMS)
    assert l2 == pytest.approx(l1, rel=1e-14)
    assert np.allclose(g1, g2, rtol=1e-13, atol=1e-16)


def test_soft_loss_at_zero_weights_is_log_k_for_any_targets():
    """Zero weights give equal logits: logsumexp = log k + z and sum_c q_c z = z."""
    P = np.zeros(oracle.mlp_nparams(*DIMS))
    X = np.random.default_rng(5).normal(size=(7, 15))
    loss, _ = oracle.mlp_loss_grad_soft(P, X, soft_targets(7, DIMS[3], 6), DIMS)
    assert loss == pytest.approx(math.log(DIMS[3]), rel=1e-15)


def test_soft_loss_minimum_is_the_targets_entropy():
    """With the last layer's bias alone set to log q (one sample), softmax(z) = q,
    the gradient in z vanishes and the loss equals the entropy of q (Gibbs)."""
    d, h1, h2, k = DIMS
    q = soft_targets(1, k, 8)[0]
    P = np.zeros(oracle.mlp_nparams(*DIMS))
    P[-k:] = np.log(q)
    loss, g = oracle.mlp_loss_grad_soft(P, np.ones((1, d)), q.reshape(1, k), DIMS)
    assert loss == pytest.approx(-np.sum(q * np.log(q)), rel=1e-12)
    assert np.allclose(g[-k:], 0.0, atol=1e-15)
