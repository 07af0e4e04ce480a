"""The Gram product Q = G G^T of the factor on the tensor cores (exact digit splitting) against
the FP64 product, and the preconditioner built from it against the oracle's inverse.

Bar: |Q - G G^T|_ij <= 1e-13 sqrt(Q_ii Q_jj) (the bound of a double-float product; each entry
is accurate to ~2^-48 of |G_i| |G_j|), identical across calls, and Q^{-1} within
1e-15 kappa(Q) m of the oracle's inverse, including a sketch with kappa(Q) >= 1e10.
"""
import numpy as np
import pytest

import synth
from oracle import hashing, iipm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def lib():
    import paper_2003_08072_gb300 as pkg

    assert torch.cuda.is_available()
    pkg.load()


def solver_for(m, tc=1, w=0):
    import paper_2003_08072_gb300 as pkg

    prm = pkg.lp_params_default()
    prm.gram_tensor_cores = tc
    prm.sketch_w = w
    lp = synth.dense_lp(0, m, max(4 * m, 64))
    return pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)


def gram_err(Q, G):
    OQ = G @ G.T
    d = np.sqrt(np.diag(OQ))
    return np.max(np.abs(Q - OQ) / np.outer(d, d))


@pytest.mark.parametrize("m,w,spread", [(37, 148, 0.0), (130, 520, 2.0), (300, 1200, 3.0),
                                        (1000, 4000, 3.0), (64, 2100, 1.0)])
def test_tensor_core_gram_matches_fp64(m, w, spread):
    """Shapes across the tile and chunk boundaries (128-row tiles, 1024-column chunks, a ragged
    last chunk), entries spread over 10^(+-spread) within rows as late in the IPM."""
    rng = np.random.default_rng(m + w)
    G = rng.standard_normal((m, w)) * 10.0 ** rng.uniform(-spread, spread, (m, w))
    G *= 10.0 ** rng.uniform(-2, 2, (m, 1))          # rows of different size
    s = solver_for(m, tc=1, w=w)
    Q1, _ = s.factor(T(np.ascontiguousarray(G.T)))
    Q2, _ = s.factor(T(np.ascontiguousarray(G.T)))
    Q1, Q2 = Q1.cpu().numpy(), Q2.cpu().numpy()
    assert gram_err(Q1, G) <= 1e-13
    assert np.array_equal(Q1, Q2)                   # no atomics: the same bits every call
    assert np.array_equal(Q1, Q1.T)
    s.close()


def test_tensor_core_and_double_float_gram_agree():
    m, w = 200, 800
    rng = np.random.default_rng(5)
    G = rng.standard_normal((m, w)) * 10.0 ** rng.uniform(-3, 3, (m, w))
    out = []
    for tc in (1, 0):
        s = solver_for(m, tc=tc, w=w)
        Q, _ = s.factor(T(np.ascontiguousarray(G.T)))
        out.append(Q.cpu().numpy())
        s.close()
    d = np.sqrt(np.diag(G @ G.T))
    assert np.max(np.abs(out[0] - out[1]) / np.outer(d, d)) <= 2e-13


def test_ill_conditioned_sketch_inverse():
    """A sketch shaped like a late IPM iterate (m "basic" columns with d over 10^(0..3), the
    others at 1e-4) with kappa(Q) >= 1e10: the inverse from the tensor-core Gram product and
    the Cholesky factor matches the oracle's within 1e-15 kappa(Q) m."""
    m, n = 120, 6000
    lp = synth.dense_lp(4, m, n)
    rng = np.random.default_rng(11)
    d = np.full(n, 1e-4)
    d[rng.choice(n, m, replace=False)] = 10.0 ** rng.uniform(0, 3.0, m)
    w = 4 * m
    b, sg = hashing.sketch_indices(0, 0, n, 4, w)
    OG = iipm.sketch_ADW(lp.A.astype(np.float64), d, b, sg, w)
    OQ = OG @ OG.T
    kappa = np.linalg.cond(OQ)
    assert kappa >= 1e10
    s = solver_for(m, tc=1)
    Q, Mi = s.factor(T(np.ascontiguousarray(OG.T)))
    Q, Mi = Q.cpu().numpy(), Mi.cpu().numpy()
    assert gram_err(Q, OG) <= 1e-13
    Oinv = np.linalg.inv(OQ)
    assert np.abs(Mi - Oinv).max() <= 1e-15 * kappa * m * np.abs(Oinv).max()
    s.close()


@pytest.mark.parametrize("tc", [1, 0])
def test_ipm_with_either_gram_matches_oracle(tc):
    import paper_2003_08072_gb300 as pkg

    lp = synth.dense_lp(0, 40, 2000)
    prm = pkg.lp_params_default()
    prm.gram_tensor_cores = tc
    s = pkg.LPSolver.dense(T(lp.At), T(lp.b), T(lp.c), params=prm)
    x, y, sv, info = s.solve()
    ref = iipm.ipm_solve(lp.A.astype(np.float64), lp.b, lp.c, iipm.Params())
    assert info.status == 0
    assert abs(info.ipm_iters - ref.iters) <= 1
    assert abs(float(lp.c @ x.cpu().numpy()) - ref.obj) <= 1e-6 * abs(ref.obj)
    s.close()
