"""l1-SVM LPs with the shape of the paper's ARCENE experiment (Table 1: 100 points, 10000
features, LP 100 x 20102) on synthetic separable Gaussian data, GPU against the oracle."""
import numpy as np
import pytest

import synth
from oracle import iipm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_arcene_shaped_svm_matches_oracle(dt):
    import paper_2003_08072_gb300 as pkg

    pts, feats = synth.SVM_SHAPES["arcene"]
    lp = synth.l1svm_lp(1, pts, feats, dtype=dt)
    A = lp.A.astype(np.float64)
    solver = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c))
    x, y, s, info = solver.solve()
    x, y, s = (t.cpu().numpy() for t in (x, y, s))
    solver.close()
    ref = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(), variant="exact")
    assert info.status == 0 and ref.converged
    assert max(iipm.kkt_scaled(A, lp.b, lp.c, x, y, s)) <= 1.01e-8
    assert abs(float(lp.c @ x) - ref.obj) <= 1e-6 * abs(ref.obj)
    assert abs(info.ipm_iters - ref.iters) <= 1, (info.ipm_iters, ref.iters)
    # the GPU's (w, b) separates the training points with margin 1
    w = x[:feats] - x[feats:2 * feats]
    b = x[2 * feats] - x[2 * feats + 1]
    margins = A[:, :feats] @ w + A[:, 2 * feats] * b
    assert margins.min() >= 1 - 1e-6
