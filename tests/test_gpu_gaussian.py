"""Gaussian sketch (Sec. 5; the sketch of the paper's experiments, Sec. 6) on the GPU against
the oracle.  Both sides generate W from the same counter (SplitMix64 uniforms, Box-Muller);
the GPU evaluates the transcendentals in FP32, so W agrees to ~1e-7 relative and the
products built from it to the same order."""
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


def make(lp, dt=np.float64):
    import paper_2003_08072_gb300 as pkg

    prm = pkg.lp_params_default()
    prm.sketch_kind = pkg._binding.LP_SKETCH_GAUSSIAN
    At = lp.At.astype(dt)
    return pkg.LPSolver.dense(T(At), T(lp.b), T(lp.c), params=prm), prm


def test_gaussian_sketch_matches_oracle():
    m, n = 40, 2000
    lp = synth.dense_lp(0, m, n)
    solver, prm = make(lp)
    x, y, s = synth.iterate_point(3, m, n, spread=3.0)
    d = np.sqrt(x / s)
    k = 5
    G = N(solver.sketch(T(d), k))
    W = hashing.gaussian_W(prm.seed, k, n, 4 * m)
    ref = lp.A @ (d[:, None] * W)
    scale = np.abs(np.abs(lp.A) @ (d[:, None] * np.abs(W))).max()
    assert np.abs(G - ref).max() <= 1e-6 * scale
    solver.close()


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
