"""Gaussian sketch (Sec. 5; the sketch of the paper's experiments, Sec. 6) on the GPU against
the oracle.  Both sides draw W from the same counter and the normal quantile table on a 2^-8
grid, computed independently (the oracle with scipy's ndtri, the library on the host by
bisection on erfc); the entries are integers over 2^8 sqrt(w), identical on both sides, so
the sketch agrees to the accuracy of the products."""
import numpy as np
import pytest

import synth
from oracle import hashing, iipm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def N(t):
    return t.detach().cpu().numpy()


def make(lp, dt=np.float64, At=None, **prm_kw):
    import paper_2003_08072_gb300 as pkg

    prm = pkg.lp_params_default()
    prm.sketch_kind = pkg._binding.LP_SKETCH_GAUSSIAN
    for k, v in prm_kw.items():
        setattr(prm, k, v)
    At = (lp.At if At is None else At).astype(dt)
    return pkg.LPSolver.dense(T(At), T(lp.b), T(lp.c), params=prm), prm


@pytest.mark.parametrize("tc", [1, 0])
@pytest.mark.parametrize("m,n,dt", [(40, 2000, np.float64), (130, 9001, np.float32),
                                    (97, 12289, np.float64)])
def test_gaussian_sketch_matches_oracle(tc, m, n, dt):
    """G = A D W on the tensor cores (exact split, tc = 1) and on the CUDA cores (double-float,
    tc = 0) against the oracle's FP64 product with the same W (integer grid values, identical
    on both sides).  The shapes cross the 4096-column chunks of the tensor-core product with a
    ragged last chunk and k block, and leave ragged tiles in m (32) and w = 4m (128); with
    n w >= 4e6 entries every cell of the quantile table is drawn."""
    lp = synth.dense_lp(0, m, n, dtype=dt)
    solver, prm = make(lp, dt, gram_tensor_cores=tc)
    x, y, s = synth.iterate_point(3, m, n, spread=3.0)
    d = np.sqrt(x / s)
    k = 5
    G = N(solver.sketch(T(d), k))
    W = hashing.gaussian_W(prm.seed, k, n, 4 * m)
    A = lp.A.astype(np.float64)
    ref = A @ (d[:, None] * W)
    scale = np.abs(np.abs(A) @ (d[:, None] * np.abs(W))).max()
    assert np.abs(G - ref).max() <= 1e-13 * scale
    solver.close()


@pytest.mark.parametrize("tc,tol", [(1, 1e-13), (0, 1e-12)])
def test_gaussian_sketch_entrywise(tc, tol):
    """Every entry of G, relative to its own scale (|A| D |W|)_ic, including a row of A D nine
    orders of magnitude below the others (its own exponent in the tensor-core split).  The
    tensor-core product is exact up to the 2^-54 digit truncation of each row of A D; the
    double-float sum on the CUDA cores accumulates n rounding errors of 2^-48."""
    m, n = 70, 6000
    lp = synth.dense_lp(2, m, n)
    x, y, s = synth.iterate_point(7, m, n, spread=6.0)
    d = np.sqrt(x / s)
    At = lp.At.copy()
    At[:, 11] *= 1e-9
    solver, prm = make(lp, np.float64, gram_tensor_cores=tc, At=At)
    G = N(solver.sketch(T(d), 3))
    solver.close()
    A = At.T
    W = hashing.gaussian_W(prm.seed, 3, n, 4 * m)
    ref = A @ (d[:, None] * W)
    absprod = np.abs(A) @ (d[:, None] * np.abs(W))
    assert np.all(np.abs(G - ref) <= tol * absprod)


def test_gaussian_normal_solve_matches_oracle():
    m, n = 40, 2000
    lp = synth.dense_lp(0, m, n)
    A = lp.A
    solver, prm = make(lp)
    x, y, s = synth.iterate_point(4, m, n, spread=3.0)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, s)
    p = iipm.rhs_p(A, lp.b, x, s, rp, rd, mu, 0.5)
    k = 2
    out = solver.normal_solve(T(x), T(s), T(p), k)
    ref = iipm.normal_solve_sketch(A, x, s, p, k, iipm.Params(sketch_kind="gaussian"))
    assert abs(out["info"].cg_iters_last - ref["cg"].iters) <= 1
    dy = N(out["dy"])
    assert np.linalg.norm(dy - ref["dy"]) <= 1e-4 * np.linalg.norm(ref["dy"])
    # Eq. addl with the GPU's own W: A S^-1 v = A D (W u) = r~
    v = np.sqrt(x * s) * N(out["Wu"])
    rt = N(out["rtil"])
    assert np.linalg.norm(A @ (v / s) - rt) <= 1e-8 * np.linalg.norm(rt) + 1e-14 * np.abs(p).max()
    solver.close()


@pytest.mark.parametrize("case", ["config1", "arcene"])
def test_gaussian_ipm_matches_oracle(case):
    if case == "config1":
        lp, dt = synth.dense_lp(0, 40, 2000), np.float64
    else:
        pts, feats = synth.SVM_SHAPES["arcene"]
        lp, dt = synth.l1svm_lp(1, pts, feats, dtype=np.float32), np.float32
    A = lp.A.astype(np.float64)
    solver, prm = make(lp, dt)
    x, y, s, info = solver.solve()
    x, y, s = N(x), N(y), N(s)
    solver.close()
    ref = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(sketch_kind="gaussian"))
    assert info.status == 0 and ref.converged
    assert max(iipm.kkt_scaled(A, lp.b, lp.c, x, y, s)) <= 1.01e-8
    assert abs(float(lp.c @ x) - ref.obj) <= 1e-6 * abs(ref.obj)
    assert abs(info.ipm_iters - ref.iters) <= 1, (info.ipm_iters, ref.iters)


def test_gaussian_sketch_needs_dense_A():
    import paper_2003_08072_gb300 as pkg

    lp = synth.sparse_lp(0, 20, 400, nnz_per_col=3)
    prm = pkg.lp_params_default()
    prm.sketch_kind = pkg._binding.LP_SKETCH_GAUSSIAN
    with pytest.raises(pkg.LPError) as e:
        pkg.LPSolver.csr(lp.m, lp.n, T(lp.indptr), T(lp.indices), T(lp.values), T(lp.b),
                         T(lp.c), params=prm)
    assert e.value.status == pkg._binding.LP_ERR_ARG
