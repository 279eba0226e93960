"""Shared pieces of the GPU parity tests (imported by tests only)."""
import numpy as np

from paper_2411_10143_b300 import workloads as W

# The configuration space the SpMV family covers.
def all_configs():
    from paper_2411_10143_b300 import cascade as C
    cfgs = [C.config("CSR", C.ALGO_SCALAR), C.config("CSR", C.ALGO_MERGE)]
    cfgs += [C.config("CSR", C.ALGO_VECTOR, tpv=t) for t in C.TPV_CLASSES]
    cfgs += [C.config("COO"), C.config("ELL")]
    cfgs += [C.config("SELL", sigma=s) for s in C.SIGMA_CLASSES]
    cfgs += [C.config("HYB", hyb_k=k) for k in (0, 1, 3)]
    cfgs += [C.config("DIA")]
    return cfgs


def ragged_matrices(int_values):
    """Small matrices spanning several tiles with ragged tails, empty rows and
    one long row; sizes the oracle handles in milliseconds."""
    rng = np.random.default_rng(42)
    out = []
    for n, m, lmax in [(1, 1, 1), (37, 41, 9), (1000, 1000, 12), (4099, 3000, 40),
                       (20000, 20000, 8)]:
        lens = rng.integers(0, lmax + 1, n)
        lens[rng.random(n) < 0.05] = 0
        if n > 100:
            lens[rng.integers(0, n)] = min(m, 2500)  # one long row
        out.append(W.random_csr(n, m, lens, seed=n, int_values=int_values))
    out.append(W.random_csr(50, 60, np.zeros(50, np.int64), seed=1, int_values=int_values))
    P = W.poisson3d(13)
    if int_values:
        P.val = np.random.default_rng(3).choice(np.array([-2.0, -1.0, 1.0, 3.0]), P.nnz)
    out.append(P)
    B = W.banded(5003, 64, 0.6, seed=9)
    if int_values:
        B.val = np.random.default_rng(4).choice(np.array([-2.0, 1.0, 2.0]), B.nnz)
    out.append(B)
    return out
