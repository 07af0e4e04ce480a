"""GPU parity of each step of the hot path against the FP64 oracle, through the C ABI.

Shapes span several column tiles, ragged row slices (m not a multiple of the 16-byte vector
or of the warp slice) and a ragged last tile (n not a multiple of the tile width).
Tolerances (FP64 unless stated): the GPU sums in a different order than numpy, so results
agree to a few units of rounding relative to the magnitude of the summed terms (1e-11).
"""
import math

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


@pytest.fixture(scope="module", autouse=True)
def lib():
    import paper_2003_08072_gb300 as pkg

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg.load()
    return pkg


CASES = [
    ("dense", 40, 2000, "f64"),
    ("dense", 37, 1999, "f32"),
    ("dense", 130, 5003, "f64"),
    ("sparse", 50, 3001, "f32"),
]


def make(kind, m, n, dt, seed=0, **prm_kw):
    import paper_2003_08072_gb300 as pkg

    prm = pkg.lp_params_default()
    for k, v in prm_kw.items():
        setattr(prm, k, v)
    if kind == "dense":
        lp = synth.dense_lp(seed, m, n, dtype=np.float32 if dt == "f32" else np.float64)
        solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
        A = lp.A.astype(np.float64)
    else:
        lp = synth.sparse_lp(seed, m, n, nnz_per_col=4)
        solver = pkg.LPSolver.csr(m, n, T(lp.indptr), T(lp.indices), T(lp.values), T(lp.b),
                                  T(lp.c), params=prm)
        A = lp.to_scipy()
    return solver, A, lp, prm


def oracle_params(prm):
    return iipm.Params(tol=prm.tol, sigma=prm.sigma, gamma=prm.gamma, cg_tol=prm.cg_rel_tol,
                       cg_max_iter=prm.cg_max_iter, sketch_s=prm.sketch_s, sketch_w=prm.sketch_w,
                       seed=prm.seed, refine_max=prm.refine_max,
                       cg_theory_rule=bool(prm.cg_theory_rule))


def close(a, b, rel, scale=None):
    scale = np.abs(b).max() if scale is None else scale
    return np.abs(a - b).max() <= rel * max(scale, 1e-300)


# ------------------------------------------------------------------ a2: sketch indices

@pytest.mark.parametrize("seed,k,n,s,w", [(0, 0, 2000, 1, 160), (7, 13, 100_003, 4, 4000),
                                          (2**63 + 5, 3, 1, 1, 8), (1, 2**31 - 1, 777, 16, 64)])
def test_sketch_indices_bit_exact(seed, k, n, s, w):
    import paper_2003_08072_gb300 as pkg

    b = torch.empty(n * s, dtype=torch.int32, device="cuda")
    sg = torch.empty(n * s, dtype=torch.int8, device="cuda")
    pkg.lp_sketch_indices(seed, k, n, s, w, b, sg)
    torch.cuda.synchronize()
    ob, osg = hashing.sketch_indices(seed, k, n, s, w)
    assert np.array_equal(N(b).reshape(n, s), ob)
    assert np.array_equal(N(sg).reshape(n, s).astype(np.float64), osg)


def test_sketch_indices_empty_and_bad():
    import paper_2003_08072_gb300 as pkg

    pkg.lp_sketch_indices(0, 0, 0, 1, 8, None, None)   # n = 0: nothing to do
    with pytest.raises(pkg.LPError):
        pkg.lp_sketch_indices(0, 0, 10, 3, 8, 1, 1)


# ------------------------------------------------------------------ a1: residuals and p

@pytest.mark.parametrize("case", CASES)
def test_residuals_and_rhs(case):
    solver, A, lp, prm = make(*case)
    m, n = case[1], case[2]
    x, y, s = synth.iterate_point(3, m, n, spread=2.0)
    rp, rd, p, mu = solver.residuals(T(x), T(y), T(s), sigma=0.5)
    orp, ord_, omu = iipm.residuals(A, lp.b, lp.c, x, y, s)
    op = iipm.rhs_p(A, lp.b, x, s, orp, ord_, omu, 0.5)
    absA = abs(A)
    scale_p = np.abs(absA @ (x + 0.5 * omu / s + (x / s) * np.abs(ord_))).max() + np.abs(lp.b).max()
    assert close(N(rp), orp, 1e-11, np.abs(absA @ x).max() + np.abs(lp.b).max())
    assert close(N(rd), ord_, 1e-11, np.abs(absA.T @ np.abs(y)).max() + np.abs(lp.c).max())
    assert close(N(p), op, 1e-11, scale_p)
    assert math.isclose(mu, omu, rel_tol=1e-12)


# ------------------------------------------------------------------ a2: sketch A D W

@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("s", [1, 2, 4, 8])
def test_sketch_matches_oracle(case, s):
    m, n = case[1], case[2]
    w = (4 * m + s - 1) // s * s        # 4m rounded up to a multiple of s
    solver, A, lp, prm = make(*case, sketch_s=s, sketch_w=w)
    x, y, sv = synth.iterate_point(5, m, n, spread=3.0)
    d = np.sqrt(x / sv)
    for k in (0, 9):
        G = N(solver.sketch(T(d), k))
        b, sg = hashing.sketch_indices(prm.seed, k, n, s, w)
        OG = iipm.sketch_ADW(A, d, b, sg, w)
        scale = np.abs(A).max() * np.abs(d).max() * max(1, n * s // w) ** 0.5 * 4
        assert G.shape == OG.shape
        assert close(G, OG, 1e-12, scale)


# ------------------------------------------------------------------ a3: factor

@pytest.mark.parametrize("case", CASES[:3])
def test_factor_matches_oracle(case):
    solver, A, lp, prm = make(*case)
    m, n = case[1], case[2]
    x, y, sv = synth.iterate_point(6, m, n, spread=3.0)
    d = np.sqrt(x / sv)
    b, sg = hashing.sketch_indices(0, 0, n, prm.sketch_s, 4 * m)
    OG = iipm.sketch_ADW(A, d, b, sg, 4 * m)
    Q, Mi = solver.factor(T(np.ascontiguousarray(OG.T)))
    Q, Mi = N(Q), N(Mi)
    OQ = OG @ OG.T
    assert close(Q, OQ, 1e-13)
    Oinv = np.linalg.inv(OQ)
    kappa = np.linalg.cond(OQ)
    assert close(Mi, Oinv, 1e-15 * kappa * m)
    assert np.allclose(Mi, Mi.T, rtol=0, atol=1e-15 * kappa * np.abs(Oinv).max())


def test_factor_flags_rank_deficient_sketch():
    import paper_2003_08072_gb300 as pkg

    solver, A, lp, prm = make("dense", 40, 600, "f64")
    G = np.random.default_rng(0).standard_normal((40, 160))
    G[7] = G[3]                     # two equal rows: rank(G) = 39
    with pytest.raises(pkg.LPError) as e:
        solver.factor(T(np.ascontiguousarray(G.T)))
    assert e.value.status == pkg._binding.LP_ERR_BREAKDOWN


@pytest.mark.parametrize("m", [40, 300, 1000, 2040])
def test_factor_one_launch_sweep_equals_block_steps(m):
    """The Cholesky sweep as one launch of tile tasks claimed in dependency order gives bitwise
    the factor of the two-launches-per-block-step sweep (each tile sees the same operations in
    the same order), on a sketch with kappa(Q) ~ 1e10; both match the inverse of G G^T.  The
    sizes give 2, 10, 32 and 64 diagonal blocks of 32 (64: the largest taking the one launch)."""
    w = 4 * m
    rng = np.random.default_rng(m)
    G = rng.standard_normal((m, w)) * np.logspace(0, -5, m)[:, None]
    out = {}
    for dag in (0, 1):
        solver, A, lp, prm = make("dense", m, 2 * m, "f64", factor_dag=dag)
        Q, Mi = solver.factor(T(np.ascontiguousarray(G.T)))
        out[dag] = (N(Q), N(Mi))
        del solver
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    OQ = G @ G.T
    kappa = np.linalg.cond(OQ)
    assert kappa > 1e9
    assert close(out[1][1], np.linalg.inv(OQ), 1e-15 * kappa * m)


def test_factor_one_launch_sweep_flags_rank_deficient_sketch():
    import paper_2003_08072_gb300 as pkg

    for dag in (0, 1):
        solver, A, lp, prm = make("dense", 300, 2000, "f64", factor_dag=dag)
        G = np.random.default_rng(1).standard_normal((300, 1200))
        G[250] = G[17]                  # rank(G) = 299: a pivot of the 8th block is lost
        with pytest.raises(pkg.LPError) as e:
            solver.factor(T(np.ascontiguousarray(G.T)))
        assert e.value.status == pkg._binding.LP_ERR_BREAKDOWN


# ------------------------------------------------------------------ a4: A D^2 A^T v

@pytest.mark.parametrize("case", CASES)
def test_normal_matvec_fp64(case):
    import paper_2003_08072_gb300 as pkg

    solver, A, lp, prm = make(*case)
    m, n = case[1], case[2]
    x, y, sv = synth.iterate_point(8, m, n, spread=4.0)
    d2 = x / sv
    v = np.random.default_rng(1).standard_normal(m)
    yv, t = solver.normal_matvec(T(d2), T(v), pkg.LP_F64, want_t=True)
    oy = iipm.normal_matvec(A, d2, v)
    absA = abs(A)
    scale = np.abs(absA @ (d2 * (absA.T @ np.abs(v)))).max()
    assert close(N(yv), oy, 1e-12, scale)
    assert close(N(t), A.T @ v, 1e-12, np.abs(absA.T @ np.abs(v)).max())


@pytest.mark.parametrize("sd", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("m,n", [(300, 20_011), (503, 9001), (2000, 6007), (5001, 5003),
                                 (8192, 8209)])
def test_normal_matvec_low_precision_stream(sd, m, n):
    """FP32 accumulation over A streamed in the given precision, against the exactly rounded
    matrix in FP64: relative error within 64 u_fp32 sqrt(m) of the |A| D^2 |A|^T |v| scale.
    The sizes span the shapes of the staged product: 1 to 4 row slices per warp, column
    groups of 8 and of 2, a ragged last group, the largest m."""
    import paper_2003_08072_gb300 as pkg

    code = pkg.DTYPE_CODES[sd]
    solver, A, lp, prm = make("dense", m, n, "f64", stream_dtype=code)
    x, y, sv = synth.iterate_point(9, m, n, spread=2.0)
    d2 = x / sv
    v = np.random.default_rng(2).standard_normal(m)
    yv = N(solver.normal_matvec(T(d2), T(v), code))
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[sd]
    Ar = torch.from_numpy(A).to(tdt).to(torch.float64).numpy()
    oy = Ar @ (d2 * (Ar.T @ v))
    scale = np.abs(abs(Ar) @ (d2 * (abs(Ar).T @ np.abs(v)))).max()
    assert np.abs(yv - oy).max() <= 64 * 2.0**-24 * math.sqrt(m) * scale


# ------------------------------------------------------------------ a4 + a5: normal solve

@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("s", [1, 4])
def test_normal_solve_matches_oracle(case, s):
    solver, A, lp, prm = make(*case, sketch_s=s)
    m, n = case[1], case[2]
    x, y, sv = synth.iterate_point(11, m, n, spread=3.0)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, sv)
    p = iipm.rhs_p(A, lp.b, x, sv, rp, rd, mu, prm.sigma)
    k = 4
    out = solver.normal_solve(T(x), T(sv), T(p), k)
    ref = iipm.normal_solve_sketch(A, x, sv, p, k, oracle_params(prm))
    it_g, it_o = out["info"].cg_iters_last, ref["cg"].iters
    fp32_cg = case[3] == "f32"      # CG products accumulate in FP32, then FP64 refinement
    dy = N(out["dy"])
    rel = np.linalg.norm(dy - ref["dy"]) / np.linalg.norm(ref["dy"])
    if fp32_cg:
        # both meet ||f|| <= target; dy agree to the CG tolerance times sqrt(kappa_pre)
        assert rel <= 1e-4, (rel, it_g, it_o)
    else:
        assert abs(it_g - it_o) <= 1
        assert rel <= (1e-9 if it_g == it_o else 1e-4), (rel, it_g, it_o)
    # r~ and A^T dy are the FP64 products of the GPU's own dy
    d2 = x / sv
    rt = iipm.normal_matvec(A, d2, dy) - p
    assert close(N(out["rtil"]), rt, 1e-10, np.abs(p).max())
    assert close(N(out["Atdy"]), A.T @ dy, 1e-12, np.abs(abs(A).T @ np.abs(dy)).max())
    # Eq. addl: A S^{-1} v = r~ with v = (XS)^{1/2} W u
    v = np.sqrt(x * sv) * N(out["Wu"])
    lhs = A @ (v / sv)
    assert np.linalg.norm(lhs - N(out["rtil"])) <= 1e-8 * np.linalg.norm(N(out["rtil"])) + 1e-14 * np.abs(p).max()
    # W u from the same hashed W
    b, sg = hashing.sketch_indices(prm.seed, k, n, s, 4 * m)
    assert close(N(out["Wu"]), iipm.apply_W(N(out["u"]), b, sg), 1e-13)
    # u = (A D W)^dagger r~ (min-norm solution) equals the oracle's for the same r~
    uo, _, _ = iipm.correction_u(ref["G"], ref["R"], N(out["rtil"]), 6)
    kG = np.linalg.cond(ref["G"])
    assert close(N(out["u"]), uo, 1e-14 * kG * kG)


def test_normal_solve_vs_exact_cholesky():
    """Per-solve accuracy: ||dy - dy*|| / ||dy*|| <= 1e-6 against the Cholesky solution."""
    import scipy.linalg as sla

    solver, A, lp, prm = make("dense", 64, 4000, "f64", cg_rel_tol=1e-9, cg_theory_rule=0)
    x, y, sv = synth.iterate_point(12, 64, 4000, spread=4.0)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, sv)
    p = iipm.rhs_p(A, lp.b, x, sv, rp, rd, mu, 0.5)
    out = solver.normal_solve(T(x), T(sv), T(p), 0)
    K = A @ ((x / sv)[:, None] * A.T)
    dstar = sla.cho_solve(sla.cho_factor(K), p)
    assert np.linalg.norm(N(out["dy"]) - dstar) <= 1e-6 * np.linalg.norm(dstar)


@pytest.mark.parametrize("sd", ["f32", "bf16"])
def test_normal_solve_low_precision_refined(sd):
    """A streamed in FP32 / BF16 inside CG, refined with FP64 residuals: the final ||f|| meets
    the same target as the FP64 path and dy matches the FP64 solve to the CG tolerance."""
    import paper_2003_08072_gb300 as pkg

    m, n = 64, 6000
    s64, A, lp, prm = make("dense", m, n, "f64")
    slo, _, _, _ = make("dense", m, n, "f64", stream_dtype=pkg.DTYPE_CODES[sd])
    x, y, sv = synth.iterate_point(13, m, n, spread=3.0)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, sv)
    p = iipm.rhs_p(A, lp.b, x, sv, rp, rd, mu, 0.5)
    o64 = s64.normal_solve(T(x), T(sv), T(p), 2)
    olo = slo.normal_solve(T(x), T(sv), T(p), 2)
    # FP64 CG stops at its target; the refined low-precision solve meets twice the target
    assert o64["info"].f_norm <= o64["info"].f_target * (1 + 1e-6)
    assert olo["info"].f_norm <= 2.0 * olo["info"].f_target
    assert abs(olo["info"].f_target - o64["info"].f_target) <= 1e-9 * o64["info"].f_target
    dy64, dylo = N(o64["dy"]), N(olo["dy"])
    assert np.linalg.norm(dylo - dy64) <= 1e-4 * np.linalg.norm(dy64)
    v = np.sqrt(x * sv) * N(olo["Wu"])
    assert np.linalg.norm(A @ (v / sv) - N(olo["rtil"])) <= 1e-8 * np.linalg.norm(N(olo["rtil"])) + 1e-14


# ------------------------------------------------------------------ a6: fused update

@pytest.mark.parametrize("case", CASES)
def test_step_matches_oracle(case):
    solver, A, lp, prm = make(*case)
    m, n = case[1], case[2]
    x, y, sv = synth.iterate_point(14, m, n, spread=1.0)
    op = oracle_params(prm)
    op.cg_tol = 1e-3
    op.cg_theory_rule = False
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, sv)
    p = iipm.rhs_p(A, lp.b, x, sv, rp, rd, mu, prm.sigma)
    sol = iipm.normal_solve_sketch(A, x, sv, p, 0, op)
    dy, Wu = sol["dy"], sol["Wu"]
    Atdy = A.T @ dy
    dx, ds, v = iipm.directions(A, x, sv, rd, mu, prm.sigma, dy, Wu)
    mu0 = mu * 1.5
    eta = 0.5 * mu / mu0
    amax, alpha, B, C = iipm.step_length(x, sv, dx, ds, prm.gamma, eta, mu0)
    xg, yg, sg = T(x), T(y), T(sv)
    gdx, gds, out = solver.step(xg, yg, sg, T(rd), T(dy), T(Atdy), T(Wu), mu, eta, mu0)
    assert close(N(gdx), dx, 1e-12, np.abs(dx).max() + np.abs(x).max())
    assert close(N(gds), ds, 1e-12, np.abs(ds).max() + np.abs(rd).max())
    assert math.isclose(out[2], B, rel_tol=1e-10, abs_tol=1e-12 * n * mu)
    assert math.isclose(out[3], C, rel_tol=1e-10, abs_tol=1e-12 * n * mu)
    assert math.isclose(out[0], amax, rel_tol=1e-10, abs_tol=1e-14)
    assert math.isclose(out[1], alpha, rel_tol=1e-10, abs_tol=1e-14)
    assert close(N(xg), x + alpha * dx, 1e-12, np.abs(x).max())
    assert close(N(sg), sv + alpha * ds, 1e-12, np.abs(sv).max() + np.abs(ds).max())
    assert close(N(yg), y + alpha * dy, 1e-12, np.abs(y).max() + np.abs(dy).max())
