"""Richardson's iteration (App. A) in place of CG on the GPU, against the oracle.

The GPU runs it in dy-space, dy += Q^-1 (p - A D^2 A^T dy), through the CG kernels with unit
step and no direction memory; the oracle in the appendix's z-space.  The sketch is made wide
(w = 40m) so that ||I - Q^-1/2 A D^2 A^T Q^-1/2|| < 1, which the appendix's analysis needs.
"""
import numpy as np
import pytest

import synth
from oracle import iipm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def N(t):
    return t.detach().cpu().numpy()


def make(m, n, w, s=4, seed=2):
    import paper_2003_08072_gb300 as pkg

    prm = pkg.lp_params_default()
    prm.inner_solver = pkg._binding.LP_INNER_RICHARDSON
    prm.sketch_w = w
    prm.sketch_s = s
    lp = synth.dense_lp(seed, m, n)
    return pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm), lp, lp.A.astype(np.float64)


def test_normal_solve_matches_oracle_richardson():
    m, n, w = 12, 3000, 480
    solver, lp, A = make(m, n, w)
    x, y, s = synth.iterate_point(5, m, n, spread=3.0)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, s)
    p = iipm.rhs_p(A, lp.b, x, s, rp, rd, mu, 0.5)
    k = 3
    out = solver.normal_solve(T(x), T(s), T(p), k)
    ref = iipm.normal_solve_sketch(A, x, s, p, k, iipm.Params(inner="richardson", sketch_w=w))
    it_g, it_o = out["info"].cg_iters_last, ref["cg"].iters
    assert abs(it_g - it_o) <= 1, (it_g, it_o)
    dy = N(out["dy"])
    rel = np.linalg.norm(dy - ref["dy"]) / np.linalg.norm(ref["dy"])
    assert rel <= (1e-9 if it_g == it_o else 1e-4), (rel, it_g, it_o)
    assert out["info"].f_norm <= out["info"].f_target * (1 + 1e-6)
    # Eq. addl holds for the Richardson direction too
    v = np.sqrt(x * s) * N(out["Wu"])
    rt = N(out["rtil"])
    assert np.linalg.norm(A @ (v / s) - rt) <= 1e-8 * np.linalg.norm(rt) + 1e-14 * np.abs(p).max()
    solver.close()


def test_ipm_with_richardson_matches_oracle():
    m, n, w = 10, 1500, 400
    solver, lp, A = make(m, n, w)
    x, y, s, info = solver.solve()
    x, y, s = N(x), N(y), N(s)
    ref = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(inner="richardson", sketch_w=w))
    assert info.status == 0 and ref.converged
    assert max(iipm.kkt_scaled(A, lp.b, lp.c, x, y, s)) <= 1.01e-8
    assert abs(float(lp.c @ x) - ref.obj) <= 1e-6 * abs(ref.obj)
    assert abs(info.ipm_iters - ref.iters) <= 1
    solver.close()


def test_diverging_richardson_is_reported_not_run_to_the_cap():
    """w = 4m CountSketch: the preconditioned spectrum passes 2, the iteration diverges, and the
    solve ends with LP_ERR_NOT_CONVERGED instead of producing a direction."""
    import paper_2003_08072_gb300 as pkg

    m, n = 12, 3000
    solver, lp, A = make(m, n, 4 * m, s=1, seed=5)
    x, y, s = synth.iterate_point(5, m, n, spread=3.0)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, s)
    p = iipm.rhs_p(A, lp.b, x, s, rp, rd, mu, 0.5)
    with pytest.raises(pkg.LPError) as e:
        solver.normal_solve(T(x), T(s), T(p), 1)
    assert e.value.status == pkg._binding.LP_ERR_NOT_CONVERGED
    assert "Richardson" in str(e.value)
    solver.close()
