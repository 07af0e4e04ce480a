"""Parity at the full benchmark sizes, in the launch configuration bench.py times.

Dense LP m=1000, n=200000 with A in FP32 (the benchmark instance) and sparse LP m=5000,
n=2,000,000 with 8 nonzeros per column (CSR, FP32 values).  Products are checked in full
against numpy/scipy FP64; sketch indices bit-exactly over all n rows; sketch columns on a
sample of buckets computed one by one from the oracle's hash; the whole IPM through the
properties that hold at any size (feasibility, duality gap, positivity) recomputed in FP64
from the GPU's final iterate.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import hashing

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def N(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def dense_case():
    import paper_2003_08072_gb300 as pkg

    assert torch.cuda.is_available()
    pkg.load()
    lp = synth.dense_lp(0, 1000, 200_000, dtype=np.float32)
    solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c))
    yield lp, solver
    solver.close()


@pytest.fixture(scope="module")
def sparse_case():
    import paper_2003_08072_gb300 as pkg

    pkg.load()
    lp = synth.sparse_lp(0, 5000, 2_000_000, nnz_per_col=8)
    solver = pkg.LPSolver.csr(lp.m, lp.n, T(lp.indptr), T(lp.indices), T(lp.values), T(lp.b),
                              T(lp.c))
    yield lp, solver
    solver.close()


def _check_products(A, solver, m, n, seed):
    import paper_2003_08072_gb300 as pkg

    x, y, s = synth.iterate_point(seed, m, n, spread=3.0)
    d2 = x / s
    v = np.random.default_rng(seed).standard_normal(m)
    t_ref = A.T @ v
    y_ref = A @ (d2 * t_ref)
    absA = abs(A)
    scale = np.abs(absA @ (d2 * (absA.T @ np.abs(v)))).max()
    # CG product: FP32 stream, FP32 accumulation
    y32 = N(solver.normal_matvec(T(d2), T(v), pkg.LP_F32))
    assert np.abs(y32 - y_ref).max() <= 64 * 2.0**-24 * math.sqrt(m) * scale
    # FP64-class product (double-float on FP32 A) with A^T v
    y64, t64 = solver.normal_matvec(T(d2), T(v), pkg.LP_F64, want_t=True)
    assert np.abs(N(y64) - y_ref).max() <= 1e-12 * scale
    assert np.abs(N(t64) - t_ref).max() <= 1e-12 * np.abs(absA.T @ np.abs(v)).max()
    return x, y, s


def _check_residuals(A, lp, solver, x, y, s):
    rp, rd, p, mu = solver.residuals(T(x), T(y), T(s), sigma=0.5)
    rp_ref = A @ x - lp.b
    rd_ref = A.T @ y + s - lp.c
    mu_ref = float(x @ s) / x.size
    g = 0.5 * mu_ref / s + (x / s) * rd_ref
    p_ref = lp.b - A @ g
    absA = abs(A)
    assert np.abs(N(rp) - rp_ref).max() <= 1e-11 * (np.abs(absA @ x).max() + np.abs(lp.b).max())
    assert np.abs(N(rd) - rd_ref).max() <= 1e-11 * (np.abs(absA.T @ np.abs(y)).max() + np.abs(lp.c).max())
    assert np.abs(N(p) - p_ref).max() <= 1e-11 * (np.abs(absA @ np.abs(g)).max() + np.abs(lp.b).max())
    assert math.isclose(mu, mu_ref, rel_tol=1e-12)


def _check_sketch(A, solver, m, n, k, sample=6):
    x, y, s = synth.iterate_point(k + 100, m, n, spread=3.0)
    d = np.sqrt(x / s)
    G = N(solver.sketch(T(d), k))
    w, sk = G.shape[1], 4
    b, sg = hashing.sketch_indices(0, k, n, sk, w)
    flat_b, flat_s = b.reshape(-1), sg.reshape(-1)
    cols = np.repeat(np.arange(n), sk)
    rng = np.random.default_rng(k)
    for bucket in rng.choice(w, size=sample, replace=False):
        members = flat_b == bucket
        ci, si = cols[members], flat_s[members]
        ref = A[:, ci] @ (si * d[ci] / math.sqrt(sk))
        ref = np.asarray(ref).ravel()
        scale = np.abs(abs(A[:, ci]) @ d[ci]).max() / math.sqrt(sk)
        assert np.abs(G[:, bucket] - ref).max() <= 1e-12 * scale


def _check_solve_invariant(A, lp, solver, m, n):
    x, y, s = synth.iterate_point(7, m, n, spread=2.0)
    rp = A @ x - lp.b
    rd = A.T @ y + s - lp.c
    mu = float(x @ s) / n
    p = lp.b - A @ (0.5 * mu / s + (x / s) * rd)
    out = solver.normal_solve(T(x), T(s), T(p), 3)
    dy, rtil = N(out["dy"]), N(out["rtil"])
    rt_ref = A @ ((x / s) * (A.T @ dy)) - p
    assert np.abs(rtil - rt_ref).max() <= 1e-10 * np.abs(p).max()
    v = np.sqrt(x * s) * N(out["Wu"])
    assert np.linalg.norm(A @ (v / s) - rtil) <= 1e-8 * np.linalg.norm(rtil) + 1e-14 * np.abs(p).max()
    assert out["info"].f_norm <= 2.0 * out["info"].f_target


class _ChunkedFP64:
    """A held in its FP32 storage (lp.At, n x m), applied in FP64 one block of columns at a
    time, so that the host never holds an FP64 copy of a multi-GB matrix."""

    def __init__(self, At, block=50_000):
        self.At, self.block = At, block

    def matvec(self, x):
        out = np.zeros(self.At.shape[1])
        for j in range(0, self.At.shape[0], self.block):
            out += self.At[j:j + self.block].astype(np.float64).T @ x[j:j + self.block]
        return out

    def rmatvec(self, y):
        return np.concatenate([self.At[j:j + self.block].astype(np.float64) @ y
                               for j in range(0, self.At.shape[0], self.block)])


def _check_ipm(A, lp, solver):
    x, y, s, info = solver.solve()
    x, y, s = N(x), N(y), N(s)
    assert info.status == 0
    Ax = A.matvec(x) if isinstance(A, _ChunkedFP64) else A @ x
    Aty = A.rmatvec(y) if isinstance(A, _ChunkedFP64) else A.T @ y
    rp = np.linalg.norm(Ax - lp.b) / (1 + np.linalg.norm(lp.b))
    rd = np.linalg.norm(Aty + s - lp.c) / (1 + np.linalg.norm(lp.c))
    gap = float(x @ s) / (1 + abs(float(lp.c @ x)))
    assert max(rp, rd, gap) <= 1.01e-8
    assert x.min() > 0 and s.min() > 0
    # weak duality: c^T x - b^T y = x^T s + x^T r_d-terms; the gap bounds the objective error
    assert abs(float(lp.c @ x) - float(lp.b @ y)) <= 1e-6 * abs(float(lp.c @ x))
    return info


def test_dense_full_sketch_indices_bit_exact():
    import paper_2003_08072_gb300 as pkg

    n, s, w = 200_000, 4, 4000
    for k in (0, 37):
        b = torch.empty(n * s, dtype=torch.int32, device="cuda")
        sg = torch.empty(n * s, dtype=torch.int8, device="cuda")
        pkg.lp_sketch_indices(0, k, n, s, w, b, sg)
        torch.cuda.synchronize()
        ob, osg = hashing.sketch_indices(0, k, n, s, w)
        assert np.array_equal(N(b).reshape(n, s), ob)
        assert np.array_equal(N(sg).reshape(n, s).astype(np.float64), osg)


def test_dense_full_products_residuals_sketch(dense_case):
    lp, solver = dense_case
    A = lp.A.astype(np.float64)
    x, y, s = _check_products(A, solver, 1000, 200_000, 1)
    _check_residuals(A, lp, solver, x, y, s)
    _check_sketch(A, solver, 1000, 200_000, 5)


def _oracle_run(name):
    """The FP64 oracle's own end-to-end run of a full-size instance, stored by
    tests/golden/make_oracle_run.py (IPM iterations, objective)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


def test_dense_full_normal_solve_and_ipm(dense_case):
    lp, solver = dense_case
    A = lp.A.astype(np.float64)
    _check_solve_invariant(A, lp, solver, 1000, 200_000)
    info = _check_ipm(A, lp, solver)
    # the oracle's own run of this very instance (same W stream, s = 4)
    ref = _oracle_run("oracle_run_dense_m1000_n200000_f32_s4.json")
    assert abs(info.ipm_iters - ref["ipm_iters"]) <= 1
    assert abs(info.obj - ref["objective"]) <= 1e-6 * abs(ref["objective"])


def test_dense_fp64_n50000_ipm_matches_oracle():
    """Config 2 with A in FP64 (n = 50000): the whole IPM on the FP64 path against the oracle's
    own run of the same instance, plus the FP64 KKT certificate."""
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(0, 1000, 50_000)
    solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c))
    info = _check_ipm(lp.A, lp, solver)
    solver.close()
    ref = _oracle_run("oracle_run_dense_m1000_n50000_f64_s4.json")
    assert abs(info.ipm_iters - ref["ipm_iters"]) <= 1
    assert abs(info.obj - ref["objective"]) <= 1e-6 * abs(ref["objective"])


def test_scaled_full_bf16_ipm_certificate():
    """Config 4 (m = 2000, n = 500000, column scales 10^U(-3,3)) with A streamed in BF16 plus
    FP64 refinement: the whole solve to the stopping rule, certified in FP64 on the host."""
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(0, 2000, 500_000, dtype=np.float32, col_scale=(-3, 3))
    prm = pkg.lp_params_default()
    prm.stream_dtype = pkg.LP_BF16
    solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
    info = _check_ipm(_ChunkedFP64(lp.At), lp, solver)
    solver.close()
    assert 20 <= info.ipm_iters <= 80


def test_sparse_full_products_residuals_sketch(sparse_case):
    lp, solver = sparse_case
    S = lp.to_scipy()
    x, y, s = _check_products(S, solver, lp.m, lp.n, 2)
    _check_residuals(S, lp, solver, x, y, s)
    _check_sketch(S.tocsc(), solver, lp.m, lp.n, 3, sample=4)


def test_sparse_full_normal_solve(sparse_case):
    lp, solver = sparse_case
    S = lp.to_scipy()
    _check_solve_invariant(S, lp, solver, lp.m, lp.n)


def test_sparse_full_ipm_certificate(sparse_case):
    """Config 3 (m = 5000, n = 2,000,000, CSR): the whole IPM, certified in FP64 on the host."""
    lp, solver = sparse_case
    info = _check_ipm(lp.to_scipy(), lp, solver)
    assert 30 <= info.ipm_iters <= 100
