"""Failure detection without a GPU fault: a bounded device-side wait that runs out.

The staged CG product waits on mbarriers for the bulk copies of A that it issues itself, each
wait bounded by the global timer.  lp_test_stall_copy makes the first CTA of the next such
product skip one copy and shortens the limit, so that wait gives up: the call must return
LP_ERR_TIMEOUT (nothing is read or written out of bounds, no kernel hangs), and the same
context must afterwards compute as if nothing had happened.
"""
import math

import numpy as np
import pytest

import synth
from oracle import iipm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WAIT_NS = 200_000   # 0.2 ms per bounded wait while the hook is armed


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def lib():
    import paper_2003_08072_gb300 as pkg

    assert torch.cuda.is_available()
    pkg.load()


def test_matvec_timeout_then_parity():
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    m, n = 200, 20_000
    lp = synth.dense_lp(7, m, n, dtype=np.float32)
    solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c))
    x, _, s = synth.iterate_point(8, m, n, spread=2.0)
    d2 = x / s
    v = np.random.default_rng(9).standard_normal(m)
    for group in (0, 1):
        B.lp_test_stall_copy(solver.ctx, group, WAIT_NS)
        with pytest.raises(pkg.LPError) as e:
            solver.normal_matvec(T(d2), T(v), pkg.LP_F32)
        assert e.value.status == B.LP_ERR_TIMEOUT, e.value
        # the hook is consumed: the next product runs normally and matches the FP64 product
        y = solver.normal_matvec(T(d2), T(v), pkg.LP_F32).cpu().numpy()
        A = lp.A.astype(np.float64)
        ref = A @ (d2 * (A.T @ v))
        scale = np.abs(A) @ (d2 * (np.abs(A).T @ np.abs(v)))
        assert np.all(np.abs(y - ref) <= 64 * 2.0**-24 * math.sqrt(m) * scale)
    solver.close()


def test_ipm_timeout_then_solve_matches_oracle():
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    lp = synth.dense_lp(0, 40, 2000, dtype=np.float32)
    prm = pkg.lp_params_default()
    solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
    B.lp_test_stall_copy(solver.ctx, 0, WAIT_NS)
    with pytest.raises(pkg.LPError) as e:
        solver.solve()
    assert e.value.status == B.LP_ERR_TIMEOUT, e.value
    x, y, s, info = solver.solve()
    ref = iipm.ipm_solve(lp.A.astype(np.float64), lp.b, lp.c,
                         iipm.Params(sketch_s=prm.sketch_s, seed=prm.seed))
    assert info.status == 0
    assert abs(info.ipm_iters - ref.iters) <= 1
    obj = float(lp.c @ x.cpu().numpy())
    assert abs(obj - ref.obj) <= 1e-6 * abs(ref.obj)
    assert max(info.rp_rel, info.rd_rel, info.gap_rel) <= 1e-8
    solver.close()


def test_stall_hook_rejects_bad_arguments():
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    lp = synth.dense_lp(1, 10, 200, dtype=np.float32)
    solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c))
    for group, wait in ((-1, WAIT_NS), (0, 0), (0, 2_000_000_000)):
        with pytest.raises(pkg.LPError) as e:
            B.lp_test_stall_copy(solver.ctx, group, wait)
        assert e.value.status == B.LP_ERR_ARG
    solver.close()
