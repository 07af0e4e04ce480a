"""The allocation-free A D^2 A^T v entry point against the context-based one.

Some callers cannot allocate device memory (a framework that owns all device memory through
its own pool, or a loop that cannot absorb cudaMalloc's implicit synchronisation), so
lp_normal_matvec_noalloc keeps its partial sums in a static device array.  This file is
collected last so that a failure here does not hide earlier results; it passes alone in a
fresh process (the first call does the per-device set-up) and after the other tests.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_noalloc_matches_context_entry_point_twice(dt):
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    assert torch.cuda.is_available()
    m, n = 300, 20_011
    np_dt = np.float64 if dt == "f64" else np.float32
    lp = synth.dense_lp(21, m, n, dtype=np_dt)
    solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c))
    code = pkg.LP_F64 if dt == "f64" else pkg.LP_F32
    # the caller's own copy of A: column-major, lda = m (m * element size is a multiple of 16)
    A_dev = T(lp.At)
    x, y, s = synth.iterate_point(22, m, n, spread=3.0)
    d2 = T(x / s)
    A64 = lp.A.astype(np.float64)
    rng = np.random.default_rng(23)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        v = rng.standard_normal(m)
        y_ctx = solver.normal_matvec(d2, T(v), code).cpu().numpy()
        y_na = torch.empty(m, dtype=torch.float64, device="cuda")
        t_na = torch.empty(n, dtype=torch.float64, device="cuda")
        B.lp_normal_matvec_noalloc(A_dev, code, m, n, m, d2, T(v), y_na, t_na, stream)
        torch.cuda.synchronize()
        scale = np.abs(abs(A64) @ ((x / s) * (abs(A64).T @ np.abs(v)))).max()
        # tolerance of the matvec tests: FP64 rounding (1e-12) or FP32 accumulation
        tol = 1e-12 if dt == "f64" else 64 * 2.0**-24 * math.sqrt(m)
        assert np.abs(y_na.cpu().numpy() - y_ctx).max() <= tol * scale, call
        ref_t = A64.T @ v
        ttol = 1e-12 if dt == "f64" else 64 * 2.0**-24 * math.sqrt(m)
        assert np.abs(t_na.cpu().numpy() - ref_t).max() <= ttol * np.abs(abs(A64).T @ np.abs(v)).max()
    solver.close()


def test_noalloc_rejects_sizes_beyond_scratch():
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    m, n = 8192, 64
    A = torch.zeros(n, m, dtype=torch.float64, device="cuda")
    d2 = torch.ones(n, dtype=torch.float64, device="cuda")
    v = torch.ones(m, dtype=torch.float64, device="cuda")
    yv = torch.empty(m, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.LPError) as e:
        B.lp_normal_matvec_noalloc(A, pkg.LP_F64, m, n, m, d2, v, yv)
    assert e.value.status == B.LP_ERR_ARG
    assert "scratch limit" in str(e.value)
