"""Checkpoint / resume of Algorithm 2 on the GPU.

A run stopped at the iteration cap and continued from (x, y, s) and its state (iteration
counter k, the start point's ||r^0|| and mu_0, the stream switch) follows the uninterrupted
run: the same W(seed, k) stream and the same neighbourhood N(gamma) (Sec. 4), so it ends after
the same total number of IPM iterations (within one: the GPU's atomic sums round differently
from run to run) at the same optimum.  The state may come from another context, as after a
restart from storage.
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


@pytest.fixture(scope="module", autouse=True)
def lib():
    import paper_2003_08072_gb300 as pkg

    assert torch.cuda.is_available()
    pkg.load()


def make(lp, **kw):
    import paper_2003_08072_gb300 as pkg

    prm = pkg.lp_params_default()
    for k, v in kw.items():
        setattr(prm, k, v)
    return pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm), prm


CASES = [("f64", "f64"), ("f32", "bf16")]


@pytest.mark.parametrize("dt,sd", CASES)
def test_resume_continues_the_run(dt, sd):
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(0, 40, 2000, dtype=np.float32 if dt == "f32" else np.float64)
    A = lp.A.astype(np.float64)
    full, _ = make(lp, stream_dtype=pkg.DTYPE_CODES[sd])
    xf, yf, sf, info_f = full.solve()
    full.close()
    assert info_f.status == 0

    stop = 12
    part, prm = make(lp, stream_dtype=pkg.DTYPE_CODES[sd], ipm_max_iter=stop)
    x, y, s, info = part.solve(check=False)
    assert info.status == pkg._binding.LP_ERR_NOT_CONVERGED and info.ipm_iters == stop
    st = part.state()
    assert st.k == stop and st.r0 > 0
    assert st.mu0 == pytest.approx(1.0, rel=1e-15)   # x = s = 1 at the start point
    prm.ipm_max_iter = 200
    part.set_params(prm)
    x2, y2, s2, info2 = part.resume(x, y, s, st)
    assert info2.status == 0
    assert abs(info2.ipm_iters - info_f.ipm_iters) <= 1, (info2.ipm_iters, info_f.ipm_iters)
    assert part.state().k == info2.ipm_iters
    x2n = N(x2)
    assert abs(float(lp.c @ x2n) - float(lp.c @ N(xf))) <= 1e-7 * abs(float(lp.c @ N(xf)))
    assert max(iipm.kkt_scaled(A, lp.b, lp.c, x2n, N(y2), N(s2))) <= 1.01e-8
    part.close()


def test_resume_from_host_checkpoint_in_new_context():
    """Checkpoint as plain host data (arrays and the four state fields), new context, host
    buffers through the C ABI."""
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    lp = synth.dense_lp(0, 40, 2000)
    ref = iipm.ipm_solve(lp.A, lp.b, lp.c, iipm.Params())
    part, prm = make(lp, ipm_max_iter=9)
    x, y, s, info = part.solve(check=False)
    saved = dict(x=N(x).copy(), y=N(y).copy(), s=N(s).copy(),
                 **{k: getattr(part.state(), k) for k in ("k", "stream_switch_iter", "r0", "mu0")})
    part.close()

    fresh, prm = make(lp)
    x, y, s = saved["x"].copy(), saved["y"].copy(), saved["s"].copy()
    st = B.lp_ipm_state(k=saved["k"], stream_switch_iter=saved["stream_switch_iter"],
                        r0=saved["r0"], mu0=saved["mu0"])
    info = B.lp_ipm_resume(fresh.ctx, x, y, s, st)
    assert info.status == 0
    assert abs(info.ipm_iters - ref.iters) <= 1, (info.ipm_iters, ref.iters)
    assert abs(float(lp.c @ x) - ref.obj) <= 1e-6 * abs(ref.obj)
    assert max(iipm.kkt_scaled(lp.A, lp.b, lp.c, x, y, s)) <= 1.01e-8
    # a state out of range is an argument error
    bad = B.lp_ipm_state(k=-1, stream_switch_iter=-1, r0=1.0, mu0=1.0)
    with pytest.raises(pkg.LPError) as e:
        B.lp_ipm_resume(fresh.ctx, x, y, s, bad)
    assert e.value.status == B.LP_ERR_ARG
    fresh.close()


def test_resume_keeps_the_stream_switch():
    """A state recording a switch to the master copy makes the resumed run stream it."""
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(0, 40, 2000, dtype=np.float32)
    part, prm = make(lp, stream_dtype=pkg.LP_BF16, ipm_max_iter=6)
    x, y, s, info = part.solve(check=False)
    st = part.state()
    if st.stream_switch_iter == -1:
        assert info.stream_dtype == pkg.LP_BF16
        st.stream_switch_iter = st.k        # as if the run had switched at its last iteration
    switched = st.stream_switch_iter
    prm.ipm_max_iter = 200
    part.set_params(prm)
    x2, y2, s2, info2 = part.resume(x, y, s, st)
    assert info2.status == 0
    assert info2.stream_dtype == pkg.LP_F32 and info2.stream_switch_iter == switched
    assert part.state().stream_switch_iter == switched
    assert max(iipm.kkt_scaled(lp.A.astype(np.float64), lp.b, lp.c, N(x2), N(y2), N(s2))) <= 1.01e-8
    part.close()
