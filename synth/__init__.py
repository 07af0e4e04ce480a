"""Seeded synthetic LP instances shared by the oracle, the tests and the benchmark.

This module only draws random numbers and assembles problem data (A, b, c).
It holds none of the interior-point method's arithmetic, so both the FP64
oracle and the CUDA path may consume its output without sharing code.

Every instance is feasible and bounded by construction (the paper's own
generator, App. D.2, does not guarantee either): a strictly positive primal
point x0 fixes b = A x0, and a strictly positive dual slack s0 with a dual
point y0 fixes c = A^T y0 + s0.  The LP is in standard form (Sec. 1, the
primal and dual problems): min c^T x s.t. A x = b, x >= 0, with m << n.

Draw order for a dense instance (numpy ``default_rng(seed)``):
  1. A, drawn column by column: ``standard_normal((n, m))`` is A^T;
  2. optional column scales 10^U(lo, hi), one per column;
  3. x0 ~ U(0.5, 1.5)^n;  4. y0 ~ N(0, 1)^m;  5. s0 ~ U(0.5, 1.5)^n.
When A is stored in float32 it is rounded BEFORE b and c are formed, so the
stored matrix is exactly the LP's matrix.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class DenseLP:
    """Dense LP.  ``At`` is A^T, shape (n, m), C-contiguous: A column-major."""

    At: np.ndarray
    b: np.ndarray
    c: np.ndarray
    x0: np.ndarray
    y0: np.ndarray
    s0: np.ndarray

    @property
    def m(self) -> int:
        return self.At.shape[1]

    @property
    def n(self) -> int:
        return self.At.shape[0]

    @property
    def A(self) -> np.ndarray:
        """A as an (m, n) view (no copy)."""
        return self.At.T


@dataclasses.dataclass
class SparseLP:
    """Sparse LP in CSR (row-compressed) form, values float32, int32 columns."""

    m: int
    n: int
    indptr: np.ndarray   # int64, length m + 1
    indices: np.ndarray  # int32 column indices, row-sorted
    values: np.ndarray   # float32
    b: np.ndarray
    c: np.ndarray
    x0: np.ndarray
    y0: np.ndarray
    s0: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.values.astype(np.float64), self.indices, self.indptr),
                             shape=(self.m, self.n))


def dense_lp(seed: int, m: int, n: int, dtype=np.float64,
             col_scale: Optional[tuple] = None) -> DenseLP:
    """Gaussian dense LP, feasible and bounded by construction.

    ``col_scale=(lo, hi)`` multiplies column j by 10^U(lo, hi) (badly scaled
    columns).  ``dtype`` is the storage type of A (float64 or float32).
    """
    rng = np.random.default_rng(seed)
    At = rng.standard_normal((n, m))
    if col_scale is not None:
        scale = 10.0 ** rng.uniform(col_scale[0], col_scale[1], n)
        At *= scale[:, None]
    At = np.ascontiguousarray(At.astype(dtype))
    x0 = rng.uniform(0.5, 1.5, n)
    y0 = rng.standard_normal(m)
    s0 = rng.uniform(0.5, 1.5, n)
    A64 = At.T.astype(np.float64)
    b = A64 @ x0
    c = A64.T @ y0 + s0
    return DenseLP(At=At, b=b, c=c, x0=x0, y0=y0, s0=s0)


def sparse_lp(seed: int, m: int, n: int, nnz_per_col: int = 8) -> SparseLP:
    """Sparse LP: each column has ``nnz_per_col`` distinct uniformly random rows.

    Column j < m always contains row j, so no row of A is empty.  Values are
    N(0, 1) rounded to float32.  Returned in CSR with int32 column indices.
    Draw order: rows (with redraws of columns holding a repeated row), values,
    then x0, y0, s0 as for the dense instance.
    """
    if nnz_per_col > m:
        raise ValueError("nnz_per_col must not exceed m")
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, m, size=(n, nnz_per_col), dtype=np.int64)
    forced = np.arange(min(m, n))
    rows[forced, 0] = forced
    while True:
        srt = np.sort(rows, axis=1)
        bad = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
        if bad.size == 0:
            break
        redraw = rng.integers(0, m, size=(bad.size, nnz_per_col), dtype=np.int64)
        keep_forced = bad < m
        redraw[keep_forced, 0] = bad[keep_forced]
        rows[bad] = redraw
    vals = rng.standard_normal(n * nnz_per_col).astype(np.float32)
    cols = np.repeat(np.arange(n, dtype=np.int64), nnz_per_col)
    rflat = rows.reshape(-1)
    order = np.lexsort((cols, rflat))
    rflat, cols, vals = rflat[order], cols[order], vals[order]
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(indptr, rflat + 1, 1)
    indptr = np.cumsum(indptr)
    x0 = rng.uniform(0.5, 1.5, n)
    y0 = rng.standard_normal(m)
    s0 = rng.uniform(0.5, 1.5, n)
    lp = SparseLP(m=m, n=n, indptr=indptr, indices=cols.astype(np.int32), values=vals,
                  b=np.zeros(m), c=np.zeros(n), x0=x0, y0=y0, s0=s0)
    S = lp.to_scipy()
    lp.b = S @ x0
    lp.c = S.T @ y0 + s0
    return lp


def sparse_to_dense_At(lp: SparseLP) -> np.ndarray:
    """A^T as a dense float64 (n, m) array (small instances only)."""
    return np.ascontiguousarray(lp.to_scipy().toarray().T)


def iterate_point(seed: int, m: int, n: int, spread: float = 0.0):
    """A positive primal-dual point (x, y, s) for testing one normal-equation solve.

    ``spread`` > 0 makes x/s range over about 10^(+-spread), imitating the
    badly scaled D of a late interior-point iteration.
    """
    rng = np.random.default_rng([seed, 7])
    x = rng.uniform(0.5, 1.5, n)
    s = rng.uniform(0.5, 1.5, n)
    y = rng.standard_normal(m)
    if spread > 0:
        e = rng.uniform(-spread, spread, n)
        x *= 10.0 ** (e / 2)
        s *= 10.0 ** (-e / 2)
    return x, y, s


def serving_requests(count: int, m_range=(16, 512), ratio_range=(20, 200), seed: int = 5):
    """Request stream: (kind, m, n, seed) per request; even index dense, odd sparse."""
    out = []
    for i in range(count):
        rng = np.random.default_rng([seed, i])
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        n = m * int(rng.integers(ratio_range[0], ratio_range[1] + 1))
        out.append(("dense" if i % 2 == 0 else "sparse", m, n, int(rng.integers(0, 2**31))))
    return out


def dense_lp_f32(seed: int, m: int, n: int) -> DenseLP:
    """Gaussian dense LP as ``dense_lp`` but with A drawn directly in float32 (faster for
    many large instances; a different random stream than ``dense_lp`` for the same seed)."""
    rng = np.random.default_rng([seed, 32])
    At = rng.standard_normal((n, m), dtype=np.float32)
    x0 = rng.uniform(0.5, 1.5, n)
    y0 = rng.standard_normal(m)
    s0 = rng.uniform(0.5, 1.5, n)
    b = x0 @ At.astype(np.float64)
    c = At.astype(np.float64) @ y0 + s0
    return DenseLP(At=At, b=b, c=c, x0=x0, y0=y0, s0=s0)


def serving_instance(kind: str, m: int, n: int, seed: int):
    """One request of the serving stream: a dense Gaussian FP32 LP, or a CSR LP at 1% density
    (max(1, round(m / 100)) nonzeros per column, column j < m holding row j)."""
    if kind == "dense":
        return dense_lp_f32(seed, m, n)
    return sparse_lp(seed, m, n, nnz_per_col=max(1, int(round(0.01 * m))))


def poisson_arrivals(count: int, rate: float, seed: int = 5) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson stream of the given rate."""
    rng = np.random.default_rng([seed, 99])
    return np.cumsum(rng.exponential(1.0 / rate, count))


# Shapes (training points, features) of the l1-SVM data sets of the paper's Table 1.
SVM_SHAPES = {"arcene": (100, 10_000), "dexter": (300, 20_000), "drivface": (606, 6_400),
              "gene_rna": (801, 20_531)}


def l1svm_lp(seed: int, points: int, features: int, dtype=np.float64) -> DenseLP:
    """Standard-form LP of an l1-regularised SVM on synthetic separable data.

    Data: x_i ~ N(0, I) in R^features, labels y_i = sign(x_i^T w* + b*) for a random w*, b*
    (separable, so the LP is feasible).  LP (points rows): variables
    [w+ (features), w- (features), b+, b-, xi (points)] >= 0,
      y_i (x_i^T (w+ - w-) + b+ - b-) - xi_i = 1,
    cost 1 on w+, w-, b+, b- (||w||_1 + |b|) and 0 on the surplus xi.  The offset is priced
    like the weights so that the optimal face stays bounded.
    x0, y0, s0 are None (the IPM starts from x = s = 1, y = 0).
    """
    rng = np.random.default_rng([seed, 11])
    X = rng.standard_normal((points, features))
    wstar = rng.standard_normal(features)
    bstar = rng.standard_normal()
    y = np.sign(X @ wstar + bstar)
    y[y == 0] = 1.0
    YX = y[:, None] * X
    A = np.concatenate([YX, -YX, y[:, None], -y[:, None], -np.eye(points)], axis=1)
    At = np.ascontiguousarray(A.T.astype(dtype))
    n = A.shape[1]
    c = np.concatenate([np.ones(2 * features + 2), np.zeros(points)])
    b = np.ones(points)
    return DenseLP(At=At, b=b, c=c, x0=None, y0=None, s0=None)
