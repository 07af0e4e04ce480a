"""A streamed below its input precision on a badly scaled LP (columns scaled by 10^U(-3,3)).

The CG products stream a 16-bit copy whose columns carry power-of-two scales folded into D^2;
FP64 refinement of the normal-equation residual wins the accuracy back, and a solve whose
refinement stops contracting streams the input-precision copy from then on.  Checked against
the FP64 oracle: the stored copy element by element (through the product), the per-iterate dy
against the exact Cholesky solution, and whole solves (iterations, objective, KKT residuals).
"""
import math

import numpy as np
import pytest

import synth
from oracle import iipm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M, NCOL = 80, 8000


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def N(t):
    return t.detach().cpu().numpy()


def solver_for(lp, sd, a_dtype="f32"):
    import paper_2003_08072_gb300 as pkg

    prm = pkg.lp_params_default()
    prm.stream_dtype = pkg.DTYPE_CODES[sd]
    At = lp.At if a_dtype == "f32" else lp.At.astype(np.float64)
    return pkg.LPSolver.dense(T(At), T(lp.b), T(lp.c), params=prm), prm


def scaled_lp(dt=np.float32):
    return synth.dense_lp(3, M, NCOL, dtype=dt, col_scale=(-3, 3))


def colscaled_copy(A, sd):
    """The stored 16-bit copy as FP64: column j rounded as A_j 2^-e_j, max |A_j| 2^-e_j in
    [0.5, 1), and scaled back by 2^e_j."""
    mx = np.abs(A).max(axis=0)
    _, e = np.frexp(mx)
    e = np.clip(np.where(mx > 0, e, 0), -60, 60)
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[sd]
    q = torch.from_numpy(A * np.ldexp(1.0, -e)[None, :]).to(tdt).to(torch.float64).numpy()
    return q * np.ldexp(1.0, e)[None, :]


@pytest.fixture(scope="module")
def trajectory():
    """Iterates of the oracle's exact-direction IPM on the scaled LP (FP32 entries)."""
    lp = scaled_lp()
    A = lp.A.astype(np.float64)
    pts = []

    def cb(k, L):
        pts.append((k, L["x"].copy(), L["y"].copy(), L["s"].copy(), L["mu"]))

    ref = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(), variant="exact", callback=cb)
    assert ref.converged
    return lp, A, ref, pts


@pytest.mark.parametrize("sd", ["bf16", "f16"])
def test_colscaled_copy_product(sd):
    """The FP32-accumulated product over the scaled copy equals A_r D^2 A_r^T v for the copy A_r
    rebuilt in FP64, within 64 u_fp32 sqrt(m) of the |A_r| D^2 |A_r|^T |v| scale."""
    import paper_2003_08072_gb300 as pkg

    lp = scaled_lp()
    A = lp.A.astype(np.float64)
    solver, _ = solver_for(lp, sd)
    x, y, s = synth.iterate_point(21, M, NCOL, spread=4.0)
    d2 = x / s
    v = np.random.default_rng(3).standard_normal(M)
    yv = N(solver.normal_matvec(T(d2), T(v), pkg.DTYPE_CODES[sd]))
    Ar = colscaled_copy(A, sd)
    oy = Ar @ (d2 * (Ar.T @ v))
    scale = np.abs(abs(Ar) @ (d2 * (abs(Ar).T @ np.abs(v)))).max()
    assert np.abs(yv - oy).max() <= 64 * 2.0**-24 * math.sqrt(M) * scale
    # the copy keeps the format's relative precision in every column, also the 10^-3 ones;
    # FP16 entries below 2^-14 of their column's scale are subnormal (absolute step 2^-24)
    u, sub = {"bf16": (2.0**-8, 0.0), "f16": (2.0**-11, 2.0**-25)}[sd]
    _, e = np.frexp(np.abs(A).max(axis=0))
    assert np.all(np.abs(Ar - A) <= u * np.abs(A) + sub * np.ldexp(1.0, e)[None, :])
    solver.close()


@pytest.mark.parametrize("sd", ["f64", "f32", "bf16", "f16"])
def test_scaled_normal_solve_per_iterate(trajectory, sd):
    """At oracle iterates early, middle and late: ||f|| = ||Q^-1/2 r~|| recomputed from the
    solve's own r~ and the oracle's sketch meets the solve's target (twice it after FP64
    refinement), and ||dy - dy*|| (dy* the exact Cholesky solution) is within the bound
    ||K^-1 Q^1/2|| ||f|| that this target implies (K = A D^2 A^T)."""
    from oracle import hashing

    lp, A, ref, pts = trajectory
    solver, prm = solver_for(lp, sd, a_dtype="f64" if sd == "f64" else "f32")
    w = 4 * M
    for k, x, y, s, mu in pts[:: max(1, len(pts) // 5)] + [pts[-1]]:
        rp, rd, _ = iipm.residuals(A, lp.b, lp.c, x, y, s)
        p = iipm.rhs_p(A, lp.b, x, s, rp, rd, mu, 0.5)
        d2 = x / s
        K = A @ (d2[:, None] * A.T)
        dstar = np.linalg.solve(K, p)
        out = solver.normal_solve(T(x), T(s), T(p), k)
        info, dy, rt = out["info"], N(out["dy"]), N(out["rtil"])
        b, sg = hashing.sketch_indices(prm.seed, k, NCOL, prm.sketch_s, w)
        G = iipm.sketch_ADW(A, np.sqrt(d2), b, sg, w)
        lam, V = np.linalg.eigh(G @ G.T)
        f = math.sqrt(float(rt @ (V @ ((V.T @ rt) / lam))))
        slack = 1.001 if sd == "f64" else 2.0
        assert f <= slack * info.f_target * (1 + 1e-5), (k, sd, f, info.f_target)
        bound = np.linalg.norm(np.linalg.solve(K, (V * np.sqrt(lam)) @ V.T), 2) * f
        err = np.linalg.norm(dy - dstar)
        assert err <= bound * (1 + 1e-6) + 1e-12 * np.linalg.norm(dstar), (k, sd, err, bound)
        # the correction keeps A S^-1 v = r~ (Eq. addl) whatever the stream
        v = np.sqrt(x * s) * N(out["Wu"])
        assert np.linalg.norm(A @ (v / s) - rt) <= 1e-8 * np.linalg.norm(rt) + 1e-14 * np.abs(p).max()
    solver.close()


@pytest.mark.parametrize("sd,a_dtype", [("f32", "f32"), ("bf16", "f32"), ("f16", "f32"),
                                        ("f64", "f64"), ("f32", "f64"), ("bf16", "f64")])
def test_scaled_ipm_matches_oracle(trajectory, sd, a_dtype):
    """Whole solve on the scaled LP: scaled KKT <= 1e-8 recomputed in FP64, objective within
    1e-6 of the oracle's, IPM iterations within 1 of the oracle's."""
    lp, A, ref, _ = trajectory
    if a_dtype == "f64":
        # the FP64 instance has its own oracle solve (b, c built from the FP64 entries)
        lp = scaled_lp(np.float64)
        A = lp.A
        ref = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(), variant="exact")
    solver, prm = solver_for(lp, sd, a_dtype)
    x, y, s, info = solver.solve()
    x, y, s = N(x), N(y), N(s)
    assert info.status == 0
    kkt = iipm.kkt_scaled(A, lp.b, lp.c, x, y, s)
    assert max(kkt) <= 1.01e-8
    assert abs(float(lp.c @ x) - ref.obj) <= 1e-6 * abs(ref.obj)
    assert abs(info.ipm_iters - ref.iters) <= 1, (info.ipm_iters, ref.iters)
    # the reported stream dtype is the one asked for unless the solve switched
    import paper_2003_08072_gb300 as pkg

    asked = pkg.DTYPE_CODES[sd] if sd != "f64" else pkg.DTYPE_CODES[a_dtype]
    if info.stream_switch_iter < 0:
        assert info.stream_dtype == asked
    else:
        assert info.stream_dtype == pkg.DTYPE_CODES[a_dtype]
        assert 0 <= info.stream_switch_iter < info.ipm_iters
    solver.close()
