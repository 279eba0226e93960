"""Seeded synthetic inputs for the solver and SpMV workloads.

This module generates matrices, right-hand-side seeds and request streams and
nothing else: it holds none of the method's arithmetic (no SpMV, no solver, no
feature or format code), so the CUDA path and the CPU oracle can both consume
its output without sharing any computation.

The paper evaluates on 22 SuiteSparse matrices (Table VI: 769 to 2.06M rows,
17.8K to 17.6M non-zeros).  Those matrices are not available here, so these
generators stand in for them with structures of the same kinds and scales:
regular stencils (3D Poisson), heavy-tailed row lengths (power law), random
uniform sparsity and banded matrices, plus SPD and nonsymmetric
(convection-diffusion) systems for CG and GMRES.

Every generator returns a :class:`Matrix` with int32 ``rowptr``/``col``
(columns strictly increasing inside each row) and float64 ``val``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Matrix:
    nrows: int
    ncols: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _from_rows_cols(n, ncols, rows, cols, vals, name) -> Matrix:
    """Assemble CSR from entries already sorted by (row, col) without duplicates."""
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=rowptr[1:])
    assert rowptr[-1] < 2**31, "int32 index range exceeded"
    return Matrix(n, ncols, rowptr.astype(np.int32), cols.astype(np.int32),
                  np.ascontiguousarray(vals, np.float64), name)


def _stencil(dims, offsets_vals, name) -> Matrix:
    """Constant-coefficient stencil on a grid with Dirichlet truncation.

    ``offsets_vals`` lists (grid offset tuple, value) pairs; entries whose
    neighbour falls outside the grid are dropped.  Grid index is row-major with
    the last dimension fastest.
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    strides = [int(np.prod(dims[i + 1:])) for i in range(len(dims))]
    coords = np.indices(dims).reshape(len(dims), -1)
    entries = []
    for off, v in offsets_vals:
        ok = np.ones(n, bool)
        for d, o in enumerate(off):
            ok &= (coords[d] + o >= 0) & (coords[d] + o < dims[d])
        shift = sum(o * s for o, s in zip(off, strides))
        entries.append((shift, v, ok))
    entries.sort(key=lambda e: e[0])  # column order inside every row
    cols = np.stack([np.arange(n) + e[0] for e in entries], axis=1)
    vals = np.stack([np.broadcast_to(np.float64(e[1]), (n,)) if np.isscalar(e[1]) else e[1]
                     for e in entries], axis=1)
    mask = np.stack([e[2] for e in entries], axis=1)
    rows = np.broadcast_to(np.arange(n)[:, None], cols.shape)
    return _from_rows_cols(n, n, rows[mask], cols[mask], vals[mask], name)


def poisson2d(N: int, values: str = "stencil", seed: int | None = None) -> Matrix:
    """5-point Laplacian on an N x N grid (4 on the diagonal, -1 off), nnz = 5N^2 - 4N.

    ``values="uniform"`` keeps the pattern but draws every value from U[-1, 1].
    """
    A = _stencil((N, N), [((0, 0), 4.0), ((-1, 0), -1.0), ((1, 0), -1.0),
                          ((0, -1), -1.0), ((0, 1), -1.0)], f"poisson2d_{N}")
    if values == "uniform":
        A.val = np.random.default_rng(seed).uniform(-1.0, 1.0, A.nnz)
    return A


def poisson3d(N: int, values: str = "stencil", seed: int | None = None) -> Matrix:
    """7-point Laplacian on an N^3 grid (6 / -1), nnz = 7N^3 - 6N^2."""
    offs = [((0, 0, 0), 6.0)]
    for d in range(3):
        for s in (-1, 1):
            o = [0, 0, 0]
            o[d] = s
            offs.append((tuple(o), -1.0))
    A = _stencil((N, N, N), offs, f"poisson3d_{N}")
    if values == "uniform":
        A.val = np.random.default_rng(seed).uniform(-1.0, 1.0, A.nnz)
    return A


def convdiff3d(N: int, peclet: float = 10.0) -> Matrix:
    """First-order upwind convection-diffusion -Lap(u) + w.grad(u) on the unit cube.

    Dirichlet boundary, h = 1/(N+1), wind w along (1, 1, 1) with cell Peclet
    number Pe = |w_d| h / 2 on every axis.  Scaled by h^2 the row is
    diag = 6 + 3 * 2Pe, upwind neighbour (index - 1 on each axis) -1 - 2Pe,
    downwind neighbour -1.  Nonsymmetric; an irreducibly diagonally dominant
    M-matrix, hence nonsingular.
    """
    offs = [((0, 0, 0), 6.0 + 3 * 2 * peclet)]
    for d in range(3):
        up = [0, 0, 0]
        up[d] = -1
        dn = [0, 0, 0]
        dn[d] = 1
        offs.append((tuple(up), -1.0 - 2 * peclet))
        offs.append((tuple(dn), -1.0))
    return _stencil((N, N, N), offs, f"convdiff3d_{N}_pe{peclet:g}")


def _zipf_lengths(rng, n, alpha, mean, lmax):
    """Row lengths from a Zipf(alpha) law truncated to [1, lmax], rescaled to ``mean``.

    The truncated law's own mean differs from the requested one (about 21 for
    alpha = 1.8, lmax = 50,000), so lengths are multiplied by mean/realised
    mean with seeded stochastic rounding and floored at 1.
    """
    k = np.arange(1, lmax + 1, dtype=np.float64)
    p = k ** (-alpha)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    raw = np.searchsorted(cdf, rng.random(n), side="right") + 1
    raw = np.minimum(raw, lmax).astype(np.float64)
    scaled = raw * (mean / raw.mean())
    lens = np.floor(scaled + rng.random(n)).astype(np.int64)
    return np.clip(lens, 1, lmax)


def _sorted_unique(key):
    """Sorted distinct values of an int64 array (sort, then drop repeats)."""
    key = np.sort(key)
    keep = np.ones(key.size, bool)
    keep[1:] = key[1:] != key[:-1]
    return key[keep]


def _random_columns(rng, lens, ncols, exclude_diag=False):
    """Distinct uniform random columns per row (duplicates drawn twice are merged)."""
    n = len(lens)
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    cols = rng.integers(0, ncols, size=rows.size, dtype=np.int64)
    if exclude_diag:
        hit = cols == rows
        cols[hit] = (cols[hit] + 1) % ncols
    key = _sorted_unique(rows * ncols + cols)
    return key // ncols, key % ncols


def powerlaw(n: int = 1_000_000, alpha: float = 1.8, mean: float = 16.0, lmax: int = 50_000,
             seed: int = 1002, longest_row: bool = True) -> Matrix:
    """Power-law row lengths (truncated Zipf, rescaled to ``mean``), uniform random columns.

    One seeded row is set to ``lmax`` entries so the maximum is reached.
    Values U[-1, 1].  The realised nnz is ``A.nnz``.
    """
    rng = np.random.default_rng(seed)
    lens = _zipf_lengths(rng, n, alpha, mean, min(lmax, n))
    if longest_row:
        lens[int(rng.integers(0, n))] = min(lmax, n)
    rows, cols = _random_columns(rng, lens, n)
    vals = rng.uniform(-1.0, 1.0, rows.size)
    return _from_rows_cols(n, n, rows, cols, vals, f"powerlaw_{n}")


def uniform_random(n: int = 2_000_000, per_row: int = 8, seed: int = 1002,
                   ncols: int | None = None) -> Matrix:
    """``per_row`` uniform random columns per row (rare duplicate draws merged), U[-1, 1]."""
    rng = np.random.default_rng(seed)
    ncols = n if ncols is None else ncols
    lens = np.full(n, per_row, np.int64)
    rows, cols = _random_columns(rng, lens, ncols)
    vals = rng.uniform(-1.0, 1.0, rows.size)
    return _from_rows_cols(n, ncols, rows, cols, vals, f"uniform_{n}x{per_row}")


def banded(n: int = 1_000_000, ndiag: int = 64, fill: float = 0.6, seed: int = 1002) -> Matrix:
    """Banded matrix: offsets -ndiag/2 .. ndiag/2 - 1; the main diagonal is always
    present, every other in-range band entry with probability ``fill``.  U[-1, 1]."""
    rng = np.random.default_rng(seed)
    offs = np.arange(-(ndiag // 2), ndiag - ndiag // 2)
    i = np.arange(n)[:, None]
    cols = i + offs[None, :]
    keep = rng.random((n, len(offs))) < fill
    keep[:, offs == 0] = True
    keep &= (cols >= 0) & (cols < n)
    rows = np.broadcast_to(i, cols.shape)[keep]
    vals = rng.uniform(-1.0, 1.0, int(keep.sum()))
    return _from_rows_cols(n, n, rows, cols[keep], vals, f"banded_{n}_{ndiag}")


def spd_powerlaw(n: int = 500_000, mean: float = 12.0, alpha: float = 1.8,
                 lmax: int | None = None, seed: int = 1003) -> Matrix:
    """Random symmetric strictly diagonally dominant (hence SPD) power-law matrix.

    Off-diagonal pattern B: Zipf(alpha) row lengths rescaled to (mean - 1)/2,
    uniform random columns, values U[-1, 1].  A = B + B^T off the diagonal
    (coincident entries summed), diag_i = sum_j |A_ij| + 1.  ``lmax`` defaults
    to n/100.
    """
    rng = np.random.default_rng(seed)
    lmax = max(2, n // 100) if lmax is None else lmax
    lens = _zipf_lengths(rng, n, alpha, (mean - 1.0) / 2.0, lmax)
    rows, cols = _random_columns(rng, lens, n, exclude_diag=True)
    vals = rng.uniform(-1.0, 1.0, rows.size)
    r2 = np.concatenate([rows, cols])
    c2 = np.concatenate([cols, rows])
    v2 = np.concatenate([vals, vals])
    k2 = r2 * n + c2
    order = np.argsort(k2, kind="stable")
    k2, v2 = k2[order], v2[order]
    first = np.ones(k2.size, bool)
    first[1:] = k2[1:] != k2[:-1]
    key = k2[first]
    v = np.add.reduceat(v2, np.flatnonzero(first)) if k2.size else np.zeros(0)
    r, c = key // n, key % n
    diag = np.zeros(n)
    np.add.at(diag, r, np.abs(v))
    diag += 1.0
    r3 = np.concatenate([r, np.arange(n)])
    c3 = np.concatenate([c, np.arange(n)])
    v3 = np.concatenate([v, diag])
    order = np.lexsort((c3, r3))
    return _from_rows_cols(n, n, r3[order], c3[order], v3[order], f"spd_powerlaw_{n}")


def diagonally_dominant(A: Matrix, margin: float = 1.0) -> Matrix:
    """Same pattern plus the diagonal, with diag_i = sum_{j != i} |A_ij| + margin.

    Turns a random-valued SpMV matrix into a nonsingular (nonsymmetric) system
    for GMRES; the input's own diagonal value, if any, is replaced.
    """
    n = A.nrows
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.rowptr))
    cols = A.col.astype(np.int64)
    off = cols != rows
    r, c, v = rows[off], cols[off], A.val[off]
    diag = np.zeros(n)
    np.add.at(diag, r, np.abs(v))
    diag += margin
    r3 = np.concatenate([r, np.arange(n)])
    c3 = np.concatenate([c, np.arange(n)])
    v3 = np.concatenate([v, diag])
    order = np.lexsort((c3, r3))
    return _from_rows_cols(n, A.ncols, r3[order], c3[order], v3[order], A.name + "_dd")


def spd_variant(A: Matrix) -> Matrix:
    """An SPD system on a square matrix's pattern, as spd_powerlaw builds one:
    the off-diagonal entries of A + A^T (coincident entries summed; the pattern
    becomes symmetric), diag_i = sum_j |off-diagonal_ij| + 1 (strict dominance,
    so CG applies)."""
    n = A.nrows
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.rowptr))
    cols = A.col.astype(np.int64)
    off = cols != rows
    r, c, v = rows[off], cols[off], A.val[off]
    r2 = np.concatenate([r, c])
    c2 = np.concatenate([c, r])
    v2 = np.concatenate([v, v])
    k2 = r2 * n + c2
    order = np.argsort(k2, kind="stable")
    k2, v2 = k2[order], v2[order]
    first = np.ones(k2.size, bool)
    first[1:] = k2[1:] != k2[:-1]
    key = k2[first]
    v = np.add.reduceat(v2, np.flatnonzero(first)) if k2.size else np.zeros(0)
    r, c = key // n, key % n
    diag = np.zeros(n)
    np.add.at(diag, r, np.abs(v))
    diag += 1.0
    r3 = np.concatenate([r, np.arange(n)])
    c3 = np.concatenate([c, np.arange(n)])
    v3 = np.concatenate([v, diag])
    order = np.lexsort((c3, r3))
    return _from_rows_cols(n, n, r3[order], c3[order], v3[order], A.name + "_spd")


def random_csr(nrows: int, ncols: int, lens, seed: int, int_values: bool = False) -> Matrix:
    """Small random CSR with given per-row lengths (capped at ncols), distinct sorted columns.

    ``int_values=True`` draws values from the integers -4..4 excluding 0, for
    which every summation order of an SpMV is exact.
    """
    rng = np.random.default_rng(seed)
    lens = np.minimum(np.asarray(lens, np.int64), ncols)
    rows_l, cols_l = [], []
    for i, L in enumerate(lens):
        c = np.sort(rng.choice(ncols, size=int(L), replace=False))
        rows_l.append(np.full(L, i))
        cols_l.append(c)
    rows = np.concatenate(rows_l) if rows_l else np.zeros(0, np.int64)
    cols = np.concatenate(cols_l) if cols_l else np.zeros(0, np.int64)
    if int_values:
        vals = rng.choice(np.array([-4, -3, -2, -1, 1, 2, 3, 4], np.float64), size=rows.size)
    else:
        vals = rng.uniform(-1.0, 1.0, rows.size)
    return _from_rows_cols(nrows, ncols, rows.astype(np.int64), cols, vals, "random")


def diag_matrix(d) -> Matrix:
    d = np.asarray(d, np.float64)
    n = len(d)
    return Matrix(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                  d.copy(), "diag")


def dense_matrix(k: int, seed: int = 0) -> Matrix:
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(k), k)
    cols = np.tile(np.arange(k), k)
    return _from_rows_cols(k, k, rows, cols, rng.uniform(-1.0, 1.0, k * k), f"dense_{k}")


def vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform vector, e.g. the exact solution x* ~ U[-1, 1]."""
    return np.random.default_rng(seed).uniform(lo, hi, n)


def int_vector(n: int, seed: int) -> np.ndarray:
    """Seeded small-integer vector (-3..3) for exact-arithmetic SpMV checks."""
    return np.random.default_rng(seed).integers(-3, 4, n).astype(np.float64)


# --------------------------------------------------------------------------- suites
MATRIX_SEED_BASE = 1000  # matrix seed = 1000 + workload index
RHS_SEED_BASE = 2000     # x* seed = 2000 + workload index


def spmv_sweep(scale: float = 1.0):
    """The four SpMV-sweep matrices: 3D Poisson 128^3 with U[-1,1] values,
    power law (n = 1M, Zipf 1.8, mean 16, max 50k), uniform (n = 2M, 8/row),
    banded (n = 1M, 64 diagonals at 60 %).  ``scale`` < 1 shrinks n for tests."""
    N3 = max(4, int(round(128 * scale ** (1 / 3))))
    return {
        "poisson3d": lambda: poisson3d(N3, values="uniform", seed=MATRIX_SEED_BASE + 1),
        "powerlaw": lambda: powerlaw(max(1000, int(1_000_000 * scale)),
                                     lmax=max(50, int(50_000 * scale)), seed=MATRIX_SEED_BASE + 1),
        "uniform": lambda: uniform_random(max(1000, int(2_000_000 * scale)), 8,
                                          seed=MATRIX_SEED_BASE + 1),
        "banded": lambda: banded(max(1000, int(1_000_000 * scale)), 64, 0.6,
                                 seed=MATRIX_SEED_BASE + 1),
    }


def training_suite(seed: int = 77, count: int = 240):
    """Varied matrices for labelling SpMV configurations (predictor training).

    Families: 2D/3D stencils, power law with several exponents and means,
    uniform random, banded with several widths and fills, block-dense rows;
    sizes log-uniform between 2^12 and 2^22 rows, so that the sizes the solver
    meets (up to about 2^21) lie inside the range rather than at its edge.
    Yields (name, builder).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        fam = i % 6
        n = int(2 ** rng.uniform(12, 22))
        s = int(rng.integers(0, 2**31 - 1))
        if fam == 0:
            N = max(8, int(round(n ** 0.5)))
            out.append((f"p2d_{N}", lambda N=N, s=s: poisson2d(N, "uniform", s)))
        elif fam == 1:
            N = max(4, int(round(n ** (1 / 3))))
            out.append((f"p3d_{N}", lambda N=N, s=s: poisson3d(N, "uniform", s)))
        elif fam == 2:
            a = float(rng.uniform(1.5, 2.6))
            m = float(rng.uniform(3, 40))
            lm = int(min(n, 2 ** rng.uniform(6, 16)))
            out.append((f"pl_{n}_{a:.2f}_{m:.1f}_{lm}",
                        lambda n=n, a=a, m=m, lm=lm, s=s: powerlaw(n, a, m, lm, s)))
        elif fam == 3:
            k = int(rng.integers(2, 48))
            out.append((f"uni_{n}_{k}", lambda n=n, k=k, s=s: uniform_random(n, k, s)))
        elif fam == 4:
            w = int(rng.choice([4, 8, 16, 32, 64, 128]))
            f = float(rng.uniform(0.2, 1.0))
            out.append((f"band_{n}_{w}_{f:.2f}", lambda n=n, w=w, f=f, s=s: banded(n, w, f, s)))
        else:
            # few dense-ish rows on a sparse background (bimodal row lengths)
            a = 1.2
            m = float(rng.uniform(4, 12))
            out.append((f"bimodal_{n}_{m:.1f}",
                        lambda n=n, a=a, m=m, s=s: powerlaw(n, a, m, min(n, 4096), s)))
    return out


def batch_suite(seed: int = 79, count: int = 240, log2_min: float = 10.0,
                log2_max: float = 15.0):
    """Small systems for labelling the batched solve's threads per row: the
    training suite's families at 2^10 to 2^15 rows (the sizes a batch holds),
    each as its SPD variant (spd_variant), so one CG batch times every pattern.
    Yields (name, builder)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        fam = i % 6
        n = int(2 ** rng.uniform(log2_min, log2_max))
        s = int(rng.integers(0, 2**31 - 1))
        if fam == 0:
            N = max(8, int(round(n ** 0.5)))
            out.append((f"p2d_{N}", lambda N=N, s=s: spd_variant(poisson2d(N, "uniform", s))))
        elif fam == 1:
            N = max(4, int(round(n ** (1 / 3))))
            out.append((f"p3d_{N}", lambda N=N, s=s: spd_variant(poisson3d(N, "uniform", s))))
        elif fam == 2:
            a = float(rng.uniform(1.5, 2.6))
            m = float(rng.uniform(3, 40))
            lm = int(min(n, 2 ** rng.uniform(6, 14)))
            out.append((f"pl_{n}_{a:.2f}_{m:.1f}_{lm}",
                        lambda n=n, a=a, m=m, lm=lm, s=s: spd_variant(powerlaw(n, a, m, lm, s))))
        elif fam == 3:
            k = int(rng.integers(2, 48))
            out.append((f"uni_{n}_{k}", lambda n=n, k=k, s=s: spd_variant(uniform_random(n, k, s))))
        elif fam == 4:
            w = int(rng.choice([4, 8, 16, 32, 64, 128]))
            f = float(rng.uniform(0.2, 1.0))
            out.append((f"band_{n}_{w}_{f:.2f}",
                        lambda n=n, w=w, f=f, s=s: spd_variant(banded(n, w, f, s))))
        else:
            m = float(rng.uniform(4, 12))
            out.append((f"bimodal_{n}_{m:.1f}",
                        lambda n=n, m=m, s=s: spd_variant(powerlaw(n, 1.2, m, min(n, 4096), s))))
    return out


# --------------------------------------------------------------------------- serving
@dataclass
class Request:
    rid: int
    arrival_s: float
    kind: str      # "poisson2d" | "poisson3d" | "spd_powerlaw" | "convdiff"
    n: int         # requested size (the generated system has about n rows)
    seed: int


def request_stream(count: int = 2000, rate_per_s: float = 100.0, nmin: float = 1e3,
                   nmax: float = 1e6, seed: int = 3000):
    """Poisson-process arrivals; n log-uniform in [nmin, nmax]; mix 40 % 2D/3D
    Poisson (half each), 30 % SPD power law, 30 % convection-diffusion."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, count))
    n = np.exp(rng.uniform(math.log(nmin), math.log(nmax), count)).astype(np.int64)
    u = rng.random(count)
    half = rng.random(count) < 0.5
    reqs = []
    for i in range(count):
        if u[i] < 0.4:
            kind = "poisson2d" if half[i] else "poisson3d"
        elif u[i] < 0.7:
            kind = "spd_powerlaw"
        else:
            kind = "convdiff"
        reqs.append(Request(i, float(t[i]), kind, int(n[i]), int(rng.integers(0, 2**31 - 1))))
    return reqs


def request_matrix(req: Request) -> Matrix:
    """The system a request solves: grid side round(n^(1/2)) or round(n^(1/3))."""
    if req.kind == "poisson2d":
        return poisson2d(max(4, int(round(req.n ** 0.5))))
    if req.kind == "poisson3d":
        return poisson3d(max(3, int(round(req.n ** (1 / 3)))))
    if req.kind == "spd_powerlaw":
        return spd_powerlaw(max(64, req.n), seed=req.seed)
    return convdiff3d(max(3, int(round(req.n ** (1 / 3)))))
