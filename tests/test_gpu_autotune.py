"""The CG product's autotuner: the launch shape it keeps is one it measured no slower than the
fixed rule, and products and solves with the tuned shape match the untuned ones."""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def lib():
    import paper_2003_08072_gb300 as pkg

    assert torch.cuda.is_available()
    pkg.load()


@pytest.mark.parametrize("stream", ["f32", "bf16"])
def test_autotuned_shape_is_measured_and_products_agree(stream):
    import paper_2003_08072_gb300 as pkg
    from paper_2003_08072_gb300 import _binding as B

    m, n = 500, 70_000                       # 140 MB of FP32 A: above the tuning threshold
    lp = synth.dense_lp(3, m, n, dtype=np.float32)
    code = pkg.DTYPE_CODES[stream]
    ys = []
    for tune in (1, 0):
        prm = pkg.lp_params_default()
        prm.autotune = tune
        prm.stream_dtype = code
        s = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
        prof = B.lp_profile_read(s.ctx)
        if tune:
            # a measured choice: either a candidate shape no slower than the fixed rule, or the
            # rule itself (ctas == 0) when no candidate beat it
            assert prof.tune_rule_us > 0 and 0 < prof.tune_us <= prof.tune_rule_us
            assert prof.tune_ctas == 0 or (prof.tune_stages >= 2 and prof.tune_tc in (2, 8))
        else:
            assert prof.tune_ctas == 0 and prof.tune_rule_us == 0
        x, _, sv = synth.iterate_point(4, m, n, spread=2.0)
        v = np.random.default_rng(5).standard_normal(m)
        ys.append(s.normal_matvec(T(x / sv), T(v), code).cpu().numpy())
        s.close()
    A = lp.A.astype(np.float64)
    if stream == "bf16":   # both products stream the same rounded, column-scaled copy
        scale = np.abs(A) @ ((x / sv) * (np.abs(A).T @ np.abs(v)))
        assert np.all(np.abs(ys[0] - ys[1]) <= 2 * 64 * 2.0**-24 * math.sqrt(m) * scale)
    else:
        ref = A @ ((x / sv) * (A.T @ v))
        scale = np.abs(A) @ ((x / sv) * (np.abs(A).T @ np.abs(v)))
        for y in ys:
            assert np.all(np.abs(y - ref) <= 64 * 2.0**-24 * math.sqrt(m) * scale)


def test_autotuned_solve_matches_fixed_rule():
    import paper_2003_08072_gb300 as pkg

    m, n = 300, 60_000
    lp = synth.dense_lp(8, m, n, dtype=np.float32)
    out = []
    for tune in (1, 0):
        prm = pkg.lp_params_default()
        prm.autotune = tune
        s = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
        x, y, sv, info = s.solve()
        out.append((float(lp.c @ x.cpu().numpy()), info))
        s.close()
    (o1, i1), (o0, i0) = out
    assert i1.status == 0 and i0.status == 0
    assert abs(i1.ipm_iters - i0.ipm_iters) <= 1
    assert abs(o1 - o0) <= 1e-6 * abs(o0)
