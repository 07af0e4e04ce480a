"""End-to-end Algorithm 2 on the GPU against the FP64 oracle and against exact optima.

Bar: IPM iteration count within one of the oracle with the same W stream, objective relative
error <= 1e-6, scaled KKT residual <= 1e-8 (the stopping rule's own tolerance).
"""
import numpy as np
import pytest

import synth
from oracle import iipm
from oracle.vertex import vertex_optimum

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def lib():
    import paper_2003_08072_gb300 as pkg

    assert torch.cuda.is_available()
    pkg.load()


def params(**kw):
    import paper_2003_08072_gb300 as pkg

    p = pkg.lp_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def oracle_params(prm):
    return iipm.Params(tol=prm.tol, sigma=prm.sigma, gamma=prm.gamma, cg_tol=prm.cg_rel_tol,
                       cg_max_iter=prm.cg_max_iter, sketch_s=prm.sketch_s, sketch_w=prm.sketch_w,
                       seed=prm.seed, cg_theory_rule=bool(prm.cg_theory_rule))


def solve_dense(lp, prm):
    import paper_2003_08072_gb300 as pkg

    s = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
    x, y, sv, info = s.solve()
    out = (x.cpu().numpy(), y.cpu().numpy(), sv.cpu().numpy(), info)
    s.close()
    return out


@pytest.mark.parametrize("dt,sd,s", [("f64", "f64", 4), ("f64", "f64", 1), ("f32", "f32", 4),
                                     ("f64", "f32", 4), ("f64", "bf16", 4), ("f64", "f64", 2),
                                     ("f32", "f32", 8)])
def test_ipm_dense_config1(dt, sd, s):
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(0, 40, 2000, dtype=np.float32 if dt == "f32" else np.float64)
    prm = params(sketch_s=s, stream_dtype=pkg.DTYPE_CODES[sd])
    x, y, sv, info = solve_dense(lp, prm)
    ref = iipm.ipm_solve(lp.A.astype(np.float64), lp.b, lp.c, oracle_params(prm))
    assert info.status == 0
    assert abs(info.ipm_iters - ref.iters) <= 1
    obj = float(lp.c @ x)
    assert abs(obj - ref.obj) <= 1e-6 * abs(ref.obj)
    assert max(info.rp_rel, info.rd_rel, info.gap_rel) <= 1e-8
    assert x.min() > 0 and sv.min() > 0


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_ipm_countsketch_two_stage_factor(dt):
    """CountSketch (s = 1, w = 4m) on a 200 x 20000 LP.  Colliding dominant columns make
    Q = (A D W)(A D W)^T numerically singular for the one-stage Gram inverse late in the path;
    the two-stage factor must keep the solve within one IPM iteration of the oracle's
    QR-based factor, to scaled KKT <= 1e-8 and the oracle's objective."""
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(0, 200, 20_000, dtype=np.float32 if dt == "f32" else np.float64)
    prm = params(sketch_s=1)
    x, y, sv, info = solve_dense(lp, prm)
    ref = iipm.ipm_solve(lp.A.astype(np.float64), lp.b, lp.c, oracle_params(prm))
    assert info.status == 0
    assert info.factor_two_stage > 0          # the case the second stage exists for
    assert abs(info.ipm_iters - ref.iters) <= 1
    assert abs(float(lp.c @ x) - ref.obj) <= 1e-6 * abs(ref.obj)
    assert max(info.rp_rel, info.rd_rel, info.gap_rel) <= 1e-8


@pytest.mark.parametrize("seed,m,n", [(1, 2, 6), (3, 4, 10), (5, 3, 9)])
def test_ipm_tiny_vs_vertex_enumeration(seed, m, n):
    lp = synth.dense_lp(seed, m, n)
    best, _ = vertex_optimum(lp.A.astype(np.float64), lp.b, lp.c)
    x, y, sv, info = solve_dense(lp, params(sketch_s=1 if m < 4 else 4))
    assert info.status == 0
    assert abs(float(lp.c @ x) - best) <= 1e-6 * max(1.0, abs(best))


def test_ipm_square_and_single_row():
    """Degenerate shapes: n = m (a single feasible point) and m = 1."""
    # CountSketch (s = 1) cannot embed an n = m problem (colliding buckets make A D W rank
    # deficient, in the oracle too), so the square case uses s = 4.
    for m, n, s in [(8, 8, 4), (1, 50, 1)]:
        lp = synth.dense_lp(2, m, n)
        x, y, sv, info = solve_dense(lp, params(sketch_s=s))
        assert info.status == 0
        ref = iipm.ipm_solve(lp.A.astype(np.float64), lp.b, lp.c, iipm.Params(sketch_s=s),
                             variant="exact")
        assert abs(float(lp.c @ x) - ref.obj) <= 1e-6 * max(1.0, abs(ref.obj))


def test_ipm_sparse():
    import paper_2003_08072_gb300 as pkg
    from scipy.optimize import linprog

    lp = synth.sparse_lp(1, 60, 5000, nnz_per_col=6)
    prm = params()
    s = pkg.LPSolver.csr(lp.m, lp.n, T(lp.indptr), T(lp.indices), T(lp.values), T(lp.b),
                         T(lp.c), params=prm)
    x, y, sv, info = s.solve()
    S = lp.to_scipy()
    ref = iipm.ipm_solve(S, lp.b, lp.c, oracle_params(prm))
    hi = linprog(lp.c, A_eq=S, b_eq=lp.b, bounds=(0, None), method="highs")
    obj = float(lp.c @ x.cpu().numpy())
    assert info.status == 0
    assert abs(info.ipm_iters - ref.iters) <= 1
    assert abs(obj - hi.fun) <= 1e-6 * abs(hi.fun)


def test_ipm_host_buffers_and_rowmajor():
    """Host (numpy) iterate buffers and a row-major host A give the same answer."""
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(4, 30, 1500)
    prm = params()
    A_row = np.ascontiguousarray(lp.A)
    s = pkg.LPSolver(30, 1500, pkg.LP_DENSE_ROWMAJOR, pkg.LP_F64, A_row, lp.b, lp.c, params=prm)
    x = np.zeros(1500)
    y = np.zeros(30)
    sv = np.zeros(1500)
    info = s.solve_host(x, y, sv)
    x2, _, _, info2 = solve_dense(lp, prm)
    assert info.status == 0 and info.ipm_iters == info2.ipm_iters
    assert np.allclose(x, x2, rtol=1e-9, atol=1e-12)


def test_invalid_inputs_fail_loudly():
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(0, 10, 100)
    bad = lp.At.copy()
    bad[5, 3] = np.nan
    with pytest.raises(pkg.LPError) as e:
        pkg.LPSolver.dense(T(bad), T(lp.b), T(lp.c))
    assert e.value.status == pkg._binding.LP_ERR_ARG
    with pytest.raises(pkg.LPError):
        bb = lp.b.copy()
        bb[0] = np.inf
        pkg.LPSolver.dense(T(lp.At), T(bb), T(lp.c))
    # rank-deficient A (two equal rows, consistent b): the paper assumes rank(A) = m; the
    # solver must either return the right optimum or report an error, never a wrong answer.
    from scipy.optimize import linprog

    At = lp.At.copy()
    At[:, 4] = At[:, 2]
    b = At.T @ lp.x0
    c = At @ lp.y0 + lp.s0
    s = pkg.LPSolver.dense(T(At), T(b), T(c))
    try:
        x, y, sv, info = s.solve()
    except pkg.LPError as e:
        assert e.status in (pkg._binding.LP_ERR_BREAKDOWN, pkg._binding.LP_ERR_NUMERIC,
                            pkg._binding.LP_ERR_NOT_CONVERGED)
    else:
        hi = linprog(c, A_eq=At.T, b_eq=b, bounds=(0, None), method="highs")
        assert abs(float(c @ x.cpu().numpy()) - hi.fun) <= 1e-6 * abs(hi.fun)


def test_iteration_cap_reports_not_converged():
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(0, 20, 400)
    s = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=params(ipm_max_iter=3))
    x, y, sv, info = s.solve(check=False)
    assert info.status == pkg._binding.LP_ERR_NOT_CONVERGED
    assert info.ipm_iters == 3
    assert np.isfinite(x.cpu().numpy()).all()


@pytest.mark.parametrize("case", ["dense_f64", "dense_f32", "dense_bf16", "sparse", "countsketch"])
def test_graph_captured_cg_matches_eager(case):
    """The device-side CG loop (one CUDA graph launch per CG solve) against the host-driven
    loop: same IPM iteration count within one, same objective to 1e-6, both to scaled KKT
    1e-8; the captured run really ran its CG solves as graphs."""
    import paper_2003_08072_gb300 as pkg

    out = {}
    for graphs in (1, 0):
        if case == "sparse":
            lp = synth.sparse_lp(1, 60, 5000, nnz_per_col=6)
            prm = params(use_graphs=graphs)
            s = pkg.LPSolver.csr(lp.m, lp.n, T(lp.indptr), T(lp.indices), T(lp.values), T(lp.b),
                                 T(lp.c), params=prm)
        else:
            dt = np.float64 if case == "dense_f64" or case == "countsketch" else np.float32
            lp = synth.dense_lp(3, 80, 6000, dtype=dt)
            prm = params(use_graphs=graphs, persistent_cg=0, sketch_s=1 if case == "countsketch" else 4,
                         stream_dtype=pkg.LP_BF16 if case == "dense_bf16" else pkg.LP_F64)
            s = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
        x, y, sv, info = s.solve()
        out[graphs] = (float(lp.c @ x.cpu().numpy()), info)
        s.close()
    (og, ig), (oe, ie) = out[1], out[0]
    assert ig.status == 0 and ie.status == 0
    assert ig.cg_graph_solves > 0 and ie.cg_graph_solves == 0
    assert abs(ig.ipm_iters - ie.ipm_iters) <= 1
    assert abs(og - oe) <= 1e-6 * abs(oe)
    assert max(ig.rp_rel, ig.rd_rel, ig.gap_rel) <= 1e-8


@pytest.mark.parametrize("case", ["dense_f32", "dense_bf16", "countsketch_f32", "wide_m"])
def test_persistent_cg_matches_eager(case):
    """The persistent CG loop (one cooperative launch per CG solve: the products and the
    preconditioner applies of all iterations in one kernel, separated by grid barriers) against
    the host-driven loop: same IPM iteration count within one, same objective to 1e-6, both to
    scaled KKT 1e-8; the persistent run really ran its CG solves that way.  CountSketch brings
    in the two-stage preconditioner (two applies per iteration), m = 1100 two row slices per
    warp in the product."""
    import paper_2003_08072_gb300 as pkg

    m, n = (1100, 12000) if case == "wide_m" else (80, 6000)
    lp = synth.dense_lp(5, m, n, dtype=np.float32)
    out = {}
    for pers in (1, 0):
        prm = params(use_graphs=0, persistent_cg=pers,
                     sketch_s=1 if case == "countsketch_f32" else 4,
                     stream_dtype=pkg.LP_BF16 if case == "dense_bf16" else pkg.LP_F64)
        s = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
        x, y, sv, info = s.solve()
        out[pers] = (float(lp.c @ x.cpu().numpy()), info)
        s.close()
    (op_, ip), (oe, ie) = out[1], out[0]
    assert ip.status == 0 and ie.status == 0
    assert ip.cg_persistent_solves > 0 and ie.cg_persistent_solves == 0
    assert abs(ip.ipm_iters - ie.ipm_iters) <= 1
    assert abs(op_ - oe) <= 1e-6 * abs(oe)
    assert max(ip.rp_rel, ip.rd_rel, ip.gap_rel) <= 1e-8
