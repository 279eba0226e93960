"""The cost-aware switch's rule (cp_gate_decide), host only: convert to the
predicted format when (iterations left) x (1 - 1/speedup) exceeds the conversion
cost in default-kernel SpMVs; iterations left extrapolate the residual decay seen
so far.  Cases with a known answer, worked by hand."""
import math

import pytest

from paper_2411_10143_b300 import cascade as C


def gate(speedup=2.0, conv_ms=5.0, spmv_ms=0.05, enabled=True):
    return C.Gate.from_dict({"speedup": [1.0] + [speedup] * 5, "conv_a_ms": [0.0] + [conv_ms] * 5,
                             "conv_b_ms": [0.0] * 6, "spmv_a_ms": spmv_ms, "spmv_b_ms": 0.0},
                            enabled=enabled)


def test_disabled_gate_always_switches():
    go, rem, cost = C.gate_decide(gate(enabled=False), C.FMT_ELL, 10**6, 10, 1.0, 0.5, 1e-10)
    assert go and rem == -1.0 and cost == -1.0


def test_fast_decay_does_not_pay_for_the_conversion():
    # residual falls 10x per iteration: from 1e-2 after 2 iterations to 1e-10
    # takes 8 more; the saving 8 * (1 - 1/2) = 4 SpMVs is below the cost 5 / 0.05 = 100
    go, rem, cost = C.gate_decide(gate(), C.FMT_ELL, 10**6, 2, 1.0, 1e-2, 1e-10)
    assert not go
    assert rem == pytest.approx(8.0, rel=1e-12) and cost == pytest.approx(100.0, rel=1e-12)


def test_slow_decay_pays_for_it():
    # 0.999 per iteration: about 23,000 iterations left, saving ~11,500 SpMVs > 100
    r = 0.999 ** 20
    go, rem, _ = C.gate_decide(gate(), C.FMT_DIA, 10**6, 20, 1.0, r, 1e-10)
    assert go and rem == pytest.approx(math.log(1e-10 / r) / math.log(0.999), rel=1e-9)


def test_break_even_is_the_cost():
    # at speedup 1.5 an iteration saves 1/3 SpMV: 299 iterations left save 99.7
    # SpMVs (below the cost of 100), 301 save 100.3 (above it)
    rate = 0.9
    r = rate ** 10
    g = gate(speedup=1.5)
    assert not C.gate_decide(g, C.FMT_HYB, 10**6, 10, 1.0, r, r * rate ** 299)[0]
    assert C.gate_decide(g, C.FMT_HYB, 10**6, 10, 1.0, r, r * rate ** 301)[0]


def test_no_history_or_no_decay_counts_as_a_long_solve():
    assert C.gate_decide(gate(), C.FMT_ELL, 10**6, 1, 1.0, 0.1, 1e-10)[0]
    go, rem, _ = C.gate_decide(gate(), C.FMT_ELL, 10**6, 10, 1.0, 1.2, 1e-10)
    assert go and rem == -1.0


def test_no_expected_gain_or_converged_keeps_the_default():
    assert not C.gate_decide(gate(speedup=1.0), C.FMT_ELL, 10**6, 10, 1.0, 0.5, 1e-10)[0]
    go, rem, _ = C.gate_decide(gate(), C.FMT_ELL, 10**6, 10, 1.0, 1e-11, 1e-10)
    assert not go and rem == 0.0


def test_cost_scales_with_the_fits():
    g = C.Gate.from_dict({"speedup": [1.0] * 6, "conv_a_ms": [0.0, 0.1, 0.2, 0.3, 0.4, 0.5],
                          "conv_b_ms": [0.0, 1.0, 2.0, 3.0, 4.0, 5.0], "spmv_a_ms": 0.01,
                          "spmv_b_ms": 0.1})
    # DIA on 2M non-zeros: (0.5 + 5 * 2) / (0.01 + 0.1 * 2) = 50 SpMVs
    _, _, cost = C.gate_decide(g, C.FMT_DIA, 2 * 10**6, 10, 1.0, 0.5, 1e-10)
    assert cost == pytest.approx(10.5 / 0.21, rel=1e-12)


def test_first_tier_uses_the_best_case_and_the_feature_cost():
    # fmt < 0 (before the feature pass): the largest speedup (4) and the cost
    # of the features plus the cheapest conversion, (0.5 + 0.25) / 0.05 = 15 SpMVs
    g = C.Gate.from_dict({"speedup": [1.0, 1.5, 4.0, 2.0, 1.2, 3.0],
                          "conv_a_ms": [0.0, 1.0, 0.25, 2.0, 0.5, 3.0], "conv_b_ms": [0.0] * 6,
                          "spmv_a_ms": 0.05, "spmv_b_ms": 0.0, "feat_a_ms": 0.5,
                          "feat_b_ms": 0.0})
    rate = 0.8
    r = rate ** 4
    # 19 iterations left save 19 * 0.75 = 14.25 SpMVs < 15; 21 save 15.75 > 15
    go, rem, cost = C.gate_decide(g, -1, 10**4, 4, 1.0, r, r * rate ** 19)
    assert not go and cost == pytest.approx(15.0, rel=1e-12)
    assert rem == pytest.approx(19.0, rel=1e-9)
    assert C.gate_decide(g, -1, 10**4, 4, 1.0, r, r * rate ** 21)[0]


# ---------------------------------------------------------------- per-matrix speedups
# cp_gate_knn_speedup: the median of format f's speedup over the k training
# matrices nearest to the matrix, in the cascade's standardised feature space.

def _knn_case(seed=5, count=40):
    import numpy as np
    rng = np.random.default_rng(seed)
    mu = rng.uniform(6.0, 9.0, 15)  # log1p(f) = mu + sd z stays positive: features are >= 0
    sd = rng.uniform(0.5, 2.0, 15)
    z = rng.standard_normal((count, 15)).astype(np.float32)
    sp = rng.uniform(0.5, 3.0, (count, 6)).astype(np.float32)
    return mu, sd, z, sp


def _features_at(z_row, mu, sd):
    """Raw features whose standardised image is z_row: log1p(f) = mu + sd z."""
    import numpy as np
    return np.expm1(mu + sd * np.asarray(z_row, np.float64))


def test_knn_speedup_on_a_training_point_with_k1_is_its_own():
    mu, sd, z, sp = _knn_case()
    for j in (0, 7, 39):
        f = _features_at(z[j], mu, sd)
        for fmt in range(6):
            got = C.gate_knn_speedup(z, sp, mu, sd, f, fmt, k=1)
            assert got == pytest.approx(float(sp[j, fmt]), rel=1e-6)


def test_knn_speedup_is_the_median_of_the_nearest():
    import numpy as np
    mu, sd, z, sp = _knn_case(seed=9)
    rng = np.random.default_rng(1)
    for trial in range(20):
        q = rng.standard_normal(15) * 0.8
        f = _features_at(q, mu, sd)
        d = ((z.astype(np.float64) - q) ** 2).sum(axis=1)
        for k in (1, 4, 7):
            near = np.argsort(d, kind="stable")[:k]
            fmt = trial % 6
            assert C.gate_knn_speedup(z, sp, mu, sd, f, fmt, k=k) == pytest.approx(
                float(np.median(sp[near, fmt].astype(np.float64))), rel=1e-6)


def test_knn_speedup_ties_go_to_the_lower_index_and_k_is_clamped():
    import numpy as np
    mu, sd = np.zeros(15), np.ones(15)
    z = np.zeros((3, 15), np.float32)  # three equidistant training points
    sp = np.array([[1, 2, 2, 2, 2, 2], [1, 4, 4, 4, 4, 4], [1, 9, 9, 9, 9, 9]], np.float32)
    f = np.zeros(15)
    assert C.gate_knn_speedup(z, sp, mu, sd, f, 1, k=1) == 2.0
    assert C.gate_knn_speedup(z, sp, mu, sd, f, 1, k=2) == 3.0   # mean of the middle two
    assert C.gate_knn_speedup(z, sp, mu, sd, f, 1, k=50) == 4.0  # k clamped to 3


def test_knn_speedup_rejects_bad_arguments():
    import numpy as np
    mu, sd, z, sp = _knn_case()
    f = np.ones(15)
    with pytest.raises(C.CascadeError):
        C.gate_knn_speedup(z, sp, mu, sd, f, 6)
    with pytest.raises(C.CascadeError):
        C.gate_knn_speedup(z, sp, mu, np.zeros(15), f, 1)
    with pytest.raises(C.CascadeError):
        C.gate_knn_speedup(z, sp, mu, sd, f, 1, k=0)


def test_shipped_neighbours_are_consistent():
    """The figures in the shipped weights: one standardised feature row and six
    speedups per training matrix, standardised with the FORMAT model's own
    mu and sd."""
    import json
    import numpy as np
    from paper_2411_10143_b300 import models
    data = json.loads(models.WEIGHTS.read_text())
    nb = data["meta"]["gate"]["neighbours"]
    z, sp = np.asarray(nb["z"]), np.asarray(nb["speedup"])
    assert z.shape[1] == 15 and sp.shape == (len(z), 6) and nb["k"] >= 1
    assert np.allclose(nb["mu"], data["stages"]["FORMAT"]["mu"])
    assert np.allclose(nb["sd"], data["stages"]["FORMAT"]["sd"])
    assert (sp >= 0).all() and np.allclose(sp[:, 0] >= 1.0 - 1e-6, True)


def test_payback_is_the_break_even_of_the_rule():
    # cost 100 SpMVs at speedup 1.5 (1/3 SpMV saved an iteration): 300 iterations
    g = gate(speedup=1.5)
    pb = C.gate_payback(g, C.FMT_HYB, 10**6)
    assert pb == pytest.approx(300.0, rel=1e-12)
    # the rule switches just above the payback and keeps just below it
    rate = 0.9
    r = rate ** 10
    assert C.gate_decide(g, C.FMT_HYB, 10**6, 10, 1.0, r, r * rate ** (pb * 1.01))[0]
    assert not C.gate_decide(g, C.FMT_HYB, 10**6, 10, 1.0, r, r * rate ** (pb * 0.99))[0]
    # a 16x format with a 2.5-SpMV conversion pays back within 2.67 iterations
    g16 = C.Gate.from_dict({"speedup": [1.0] + [16.0] * 5, "conv_a_ms": [0.0] + [0.125] * 5,
                            "conv_b_ms": [0.0] * 6, "spmv_a_ms": 0.05, "spmv_b_ms": 0.0})
    assert C.gate_payback(g16, C.FMT_HYB, 10**6) == pytest.approx(2.5 / (1 - 1 / 16), rel=1e-12)


def test_payback_without_gain_or_without_the_rule():
    assert C.gate_payback(gate(speedup=1.0), C.FMT_ELL, 10**6) == math.inf
    assert C.gate_payback(gate(enabled=False), C.FMT_ELL, 10**6) == 0.0
    assert C.gate_payback(gate(), C.FMT_CSR, 10**6) == 0.0


def test_first_tier_payback_takes_the_best_case_and_the_features():
    g = C.Gate.from_dict({"speedup": [1.0, 1.2, 3.0, 1.1, 1.1, 1.1],
                          "conv_a_ms": [0.0, 1.0, 4.0, 0.5, 2.0, 2.0], "conv_b_ms": [0.0] * 6,
                          "spmv_a_ms": 0.1, "spmv_b_ms": 0.0, "feat_a_ms": 0.5, "feat_b_ms": 0.0})
    # best speedup 3 (1/3 kept), cheapest conversion 0.5 ms + features 0.5 ms = 10 SpMVs
    assert C.gate_payback(g, -1, 10**6) == pytest.approx(10.0 / (1 - 1 / 3), rel=1e-12)
