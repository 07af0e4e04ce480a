"""Pins of the FP64 oracle (oracle/iipm.py) to facts the paper and mathematics fix.

Each test checks the oracle against something other than itself: an exact
optimum found by vertex enumeration, a library LP solver, an algebraic
identity of Sec. 3-4 / App. C, an independent route through Alg. 1 (SVD and
plain CG), or brute force on tiny inputs.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import hashing, iipm
from oracle.vertex import vertex_optimum


# ------------------------------------------------------------------ P1 / P2

@pytest.mark.parametrize("seed,m,n", [(1, 2, 6), (2, 3, 8), (3, 4, 10), (4, 3, 9), (5, 2, 10)])
@pytest.mark.parametrize("variant", ["exact", "sketch"])
def test_ipm_matches_vertex_enumeration(seed, m, n, variant):
    """P1: the IIPM optimum equals the best basic feasible solution."""
    lp = synth.dense_lp(seed, m, n)
    A = lp.A.astype(np.float64)
    best, _ = vertex_optimum(A, lp.b, lp.c)
    r = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(sketch_s=1 if m < 4 else 4), variant=variant)
    assert r.converged
    assert abs(r.obj - best) <= 1e-6 * max(1.0, abs(best))
    assert r.kkt <= 1e-8


def test_ipm_matches_highs_config1():
    """P2: objective of the m=40, n=2000 Gaussian LP against SciPy HiGHS."""
    from scipy.optimize import linprog

    lp = synth.dense_lp(0, 40, 2000)
    A = lp.A.astype(np.float64)
    hi = linprog(lp.c, A_eq=A, b_eq=lp.b, bounds=(0, None), method="highs")
    assert hi.status == 0
    ex = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(), variant="exact")
    for s in (1, 4):
        sk = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(sketch_s=s), variant="sketch")
        assert sk.converged and sk.kkt <= 1e-8
        assert abs(sk.obj - hi.fun) <= 1e-6 * abs(hi.fun)
        assert abs(sk.iters - ex.iters) <= 1
    assert abs(ex.obj - hi.fun) <= 1e-6 * abs(hi.fun)


def test_sparse_lp_matches_highs():
    """P2 on a small CSR instance of the sparse generator."""
    from scipy.optimize import linprog

    lp = synth.sparse_lp(0, 30, 900, nnz_per_col=4)
    S = lp.to_scipy()
    hi = linprog(lp.c, A_eq=S, b_eq=lp.b, bounds=(0, None), method="highs")
    r = iipm.ipm_solve(S, lp.b, lp.c, iipm.Params(), variant="sketch")
    assert r.converged
    assert abs(r.obj - hi.fun) <= 1e-6 * abs(hi.fun)


# ------------------------------------------------------------------ A2

def test_rhs_literal_equals_simplified():
    """Eq. pdef written term by term equals b - A(sigma mu/s + d^2 r_d)."""
    lp = synth.dense_lp(7, 12, 300)
    A = lp.A.astype(np.float64)
    x, y, s = synth.iterate_point(7, 12, 300, spread=2)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, s)
    p1 = iipm.rhs_p(A, lp.b, x, s, rp, rd, mu, 0.5)
    p2 = iipm.rhs_p_short(A, lp.b, x, s, rd, mu, 0.5)
    assert np.allclose(p1, p2, rtol=1e-10, atol=1e-10 * np.abs(p1).max())


def test_p_is_the_exact_newton_rhs():
    """With v = 0 and exact dy, the direction solves the Newton system (Eq. system)."""
    lp = synth.dense_lp(8, 10, 200)
    A = lp.A.astype(np.float64)
    x, y, s = synth.iterate_point(8, 10, 200)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, s)
    p = iipm.rhs_p(A, lp.b, x, s, rp, rd, mu, 0.5)
    K = A @ ((x / s)[:, None] * A.T)
    dy = np.linalg.solve(K, p)
    dx, ds, v = iipm.directions(A, x, s, rd, mu, 0.5, dy, np.zeros(200))
    # the three blocks of the Newton system of the perturbed KKT conditions
    assert np.allclose(A @ dx, -rp, atol=1e-9 * np.abs(rp).max())
    assert np.allclose(A.T @ dy + ds, -rd, atol=1e-12)
    assert np.allclose(s * dx + x * ds, -x * s + 0.5 * mu, atol=1e-12)


# ------------------------------------------------------------------ sketch

def test_sketch_equals_dense_W_product():
    """The scatter form of A D W equals A D W with W materialised (dense and CSR A)."""
    lp = synth.dense_lp(2, 9, 500)
    A = lp.A.astype(np.float64)
    d = np.random.default_rng(2).uniform(0.1, 3, 500)
    for s in (1, 4):
        b, sg = hashing.sketch_indices(4, 2, 500, s, 36)
        W = iipm.sketch_W_dense(b, sg, 36)
        G = iipm.sketch_ADW(A, d, b, sg, 36)
        assert np.allclose(G, A @ np.diag(d) @ W, atol=1e-12)
        sp = synth.sparse_lp(3, 9, 500, nnz_per_col=3)
        S = sp.to_scipy()
        Gs = iipm.sketch_ADW(S, d, b, sg, 36)
        assert np.allclose(Gs, S.toarray() @ np.diag(d) @ W, atol=1e-12)
        u = np.random.default_rng(1).standard_normal(36)
        assert np.allclose(iipm.apply_W(u, b, sg), W @ u, atol=1e-13)


# ------------------------------------------------------------------ P3 / P4 / P5 / P6

def _setup(seed=0, m=20, n=800, spread=3.0, s=4, w=None):
    lp = synth.dense_lp(seed, m, n)
    A = lp.A.astype(np.float64)
    x, y, sv = synth.iterate_point(seed, m, n, spread=spread)
    w = w or 4 * m
    b, sg = hashing.sketch_indices(seed, 0, n, s, w)
    d2 = x / sv
    G = iipm.sketch_ADW(A, np.sqrt(d2), b, sg, w)
    return lp, A, x, y, sv, d2, G, b, sg


def test_factor_reproduces_Q():
    lp, A, x, y, s, d2, G, b, sg = _setup()
    R = iipm.factor_R(G)
    Q = G @ G.T
    assert np.allclose(R.T @ R, Q, rtol=0, atol=1e-12 * np.abs(Q).max())
    assert np.allclose(np.triu(R), R)


def test_pcg_equals_cg_on_precond_alt_and_rho_is_f_norm():
    """P3: PCG(M=Q) and CG on Eq. precond_alt with Q^{-1/2} from the SVD give the same dy,
    and rho_j equals ||f^(j)||^2 with f^(j) = Q^{-1/2} (A D^2 A^T dy_j - p)."""
    lp, A, x, y, s, d2, G, b, sg = _setup()
    p = np.random.default_rng(1).standard_normal(A.shape[0])
    R = iipm.factor_R(G)
    mv = lambda v: iipm.normal_matvec(A, d2, v)
    Qmh = iipm.q_inv_half_svd(G)
    res1 = iipm.pcg(mv, p, lambda r: iipm.q_inverse_apply(R, r), 1e-10, 200)
    res2 = iipm.cg_precond_alt(mv, p, Qmh, 1e-10, 200)
    assert res1.iters == res2.iters
    assert np.allclose(res1.dy, res2.dy, rtol=1e-8, atol=1e-10 * np.abs(res1.dy).max())
    assert np.allclose(res1.rho, res2.rho, rtol=1e-6, atol=1e-20)
    # rho_j = ||f^(j)||^2 recomputed from explicit iterates (truncated runs)
    for t in (1, 3, 6):
        rt = iipm.pcg(mv, p, lambda r: iipm.q_inverse_apply(R, r), 0.0, t)
        f = Qmh @ (mv(rt.dy) - p)
        assert math.isclose(rt.rho[-1], float(f @ f), rel_tol=1e-7)
    # exact solution: Cholesky of A D^2 A^T
    K = A @ (d2[:, None] * A.T)
    dstar = sla.cho_solve(sla.cho_factor(K), p)
    assert np.linalg.norm(res1.dy - dstar) <= 1e-7 * np.linalg.norm(dstar)


def test_preconditioned_spectrum_identity_and_lemma31():
    """P4: eig(Q^{-1/2} A D^2 A^T Q^{-1/2}) = 1 / eig(V^T W W^T V) (proof of Lemma 3.1),
    and when eps = ||V^T W W^T V - I|| < 1 the spectrum lies in [1/(1+eps), 1/(1-eps)]."""
    lp, A, x, y, s, d2, G, b, sg = _setup(w=4 * 20 * 8)
    w = G.shape[1]
    W = iipm.sketch_W_dense(b, sg, w)
    AD = A * np.sqrt(d2)[None, :]
    _, _, Vt = np.linalg.svd(AD, full_matrices=False)
    M = Vt @ W @ W.T @ Vt.T
    ev_m = np.sort(np.linalg.eigvalsh(M))
    Qmh = iipm.q_inv_half_svd(G)
    P = Qmh @ (AD @ AD.T) @ Qmh
    ev_p = np.sort(np.linalg.eigvalsh((P + P.T) / 2))
    assert np.allclose(np.sort(1.0 / ev_m), ev_p, rtol=1e-8)
    eps = np.abs(np.linalg.eigvalsh(M - np.eye(M.shape[0]))).max()
    if eps < 1:
        assert ev_p.min() >= 1 / (1 + eps) - 1e-10 and ev_p.max() <= 1 / (1 - eps) + 1e-10


def test_cg_residual_decay_when_well_conditioned():
    """P5: with kappa_pre < 3, ||f^(j)|| <= (kappa_pre - 1)/2 ||f^(j-1)|| (Lemma 3.2, Eq. rec)."""
    m, n = 15, 3000
    lp = synth.dense_lp(11, m, n)
    A = lp.A.astype(np.float64)
    x, y, s = synth.iterate_point(11, m, n, spread=4)
    d2 = x / s
    rng = np.random.default_rng(3)
    w = 60 * m
    W = rng.standard_normal((n, w)) / math.sqrt(w)   # Gaussian sketch (Sec. 5)
    G = iipm.sketch_ADW_given_W(A, np.sqrt(d2), W)
    Qmh = iipm.q_inv_half_svd(G)
    AD = A * np.sqrt(d2)[None, :]
    P = Qmh @ AD @ AD.T @ Qmh
    ev = np.linalg.eigvalsh((P + P.T) / 2)
    kappa = ev.max() / ev.min()
    assert kappa < 3
    R = iipm.factor_R(G)
    p = rng.standard_normal(m)
    res = iipm.pcg(lambda v: iipm.normal_matvec(A, d2, v), p,
                   lambda r: iipm.q_inverse_apply(R, r), 1e-12, 50)
    f = np.sqrt(np.maximum(res.rho, 0))
    for j in range(1, len(f)):
        assert f[j] <= (kappa - 1) / 2 * f[j - 1] * (1 + 1e-6) + 1e-14 * f[0]


def test_gaussian_sketch_condition_matches_marchenko_pastur():
    """P6: for Gaussian W, kappa_pre ~ kappa of an m x w Gaussian Gram matrix, whose
    edge ratio ((1+sqrt(m/w))/(1-sqrt(m/w)))^2 reproduces Table 1's kappa_Sk column
    (34.0 / 62.0 predicted vs 38.09 / 75.42 printed for ARCENE / DEXTER sizes)."""
    rng = np.random.default_rng(5)
    for m, w, printed in [(100, 200, 38.09), (300, 500, 75.42)]:
        pred = ((1 + math.sqrt(m / w)) / (1 - math.sqrt(m / w))) ** 2
        # rotation invariance: V^T W is exactly an m x w Gaussian, whatever A and D are
        ks = []
        for _ in range(3):
            Z = rng.standard_normal((m, w))
            ev = np.linalg.eigvalsh(Z @ Z.T)
            ks.append(ev.max() / ev.min())
        k = float(np.median(ks))
        assert 0.8 * pred <= k <= 1.6 * pred
        assert 0.8 * pred <= printed <= 1.6 * pred
    # and the same kappa through an actual A D (small case, exact identity of P4)
    m, n, w = 20, 1500, 40
    lp = synth.dense_lp(12, m, n)
    A = lp.A.astype(np.float64)
    x, y, s = synth.iterate_point(12, m, n, spread=3)
    d = np.sqrt(x / s)
    W = rng.standard_normal((n, w))
    G = iipm.sketch_ADW_given_W(A, d, W)
    AD = A * d[None, :]
    _, _, Vt = np.linalg.svd(AD, full_matrices=False)
    ev1 = np.linalg.eigvalsh(Vt @ W @ W.T @ Vt.T)
    Qmh = iipm.q_inv_half_svd(G)
    P = Qmh @ AD @ AD.T @ Qmh
    ev2 = np.linalg.eigvalsh((P + P.T) / 2)
    assert math.isclose(ev1.max() / ev1.min(), ev2.max() / ev2.min(), rel_tol=1e-7)


# ------------------------------------------------------------------ P7 / P8 / P9

def _one_iteration(seed=0, m=20, n=800, spread=2.0, s=4, cg_tol=1e-3):
    lp = synth.dense_lp(seed, m, n)
    A = lp.A.astype(np.float64)
    x, y, sv = synth.iterate_point(seed, m, n, spread=spread)
    prm = iipm.Params(sketch_s=s, cg_tol=cg_tol, cg_theory_rule=False)
    rp, rd, mu = iipm.residuals(A, lp.b, lp.c, x, y, sv)
    p = iipm.rhs_p(A, lp.b, x, sv, rp, rd, mu, prm.sigma)
    sol = iipm.normal_solve_sketch(A, x, sv, p, 0, prm)
    dx, ds, v = iipm.directions(A, x, sv, rd, mu, prm.sigma, sol["dy"], sol["Wu"])
    return dict(lp=lp, A=A, x=x, y=y, s=sv, rp=rp, rd=rd, mu=mu, p=p, sol=sol, dx=dx, ds=ds,
                v=v, prm=prm)


def test_correction_vector_invariants():
    """P7: A S^{-1} v = A D^2 A^T dy - p (Eq. addl) and the system of Eq. iip_3 hold,
    even though CG stopped early (loose tolerance)."""
    for s in (1, 4):
        it = _one_iteration(s=s)
        A, x, sv, v = it["A"], it["x"], it["s"], it["v"]
        rtil = it["sol"]["rtil"]
        assert np.linalg.norm(rtil) > 1e-6 * np.linalg.norm(it["p"])  # really inexact
        lhs = A @ (v / sv)
        assert np.linalg.norm(lhs - rtil) <= 1e-10 * np.linalg.norm(rtil)
        assert np.allclose(A @ it["dx"], -it["rp"], atol=1e-9 * np.abs(it["rp"]).max())
        assert np.allclose(A.T @ it["sol"]["dy"] + it["ds"], -it["rd"], atol=1e-12)
        mu, sig = it["mu"], it["prm"].sigma
        assert np.allclose(sv * it["dx"] + x * it["ds"], -x * sv + sig * mu - v,
                           atol=1e-12 * max(1, np.abs(x * sv).max()))


def test_residuals_shrink_linearly_after_step():
    """r(alpha) = (1 - alpha) r after a corrected step (App. C, from Eq. iip_3)."""
    it = _one_iteration()
    A, lp = it["A"], it["lp"]
    for a in (0.25, 0.7):
        x2 = it["x"] + a * it["dx"]
        y2 = it["y"] + a * it["sol"]["dy"]
        s2 = it["s"] + a * it["ds"]
        rp2, rd2, _ = iipm.residuals(A, lp.b, lp.c, x2, y2, s2)
        assert np.allclose(rp2, (1 - a) * it["rp"], atol=1e-9 * np.abs(it["rp"]).max())
        assert np.allclose(rd2, (1 - a) * it["rd"], atol=1e-11 * np.abs(it["rd"]).max())


def test_mu_linear_coefficient_closed_form():
    """P8: x^T ds + s^T dx = -(1 - sigma) n mu - 1^T v (sum of Eq. iip_3_3)."""
    it = _one_iteration()
    n = it["x"].size
    B = it["x"] @ it["ds"] + it["s"] @ it["dx"]
    want = -(1 - it["prm"].sigma) * n * it["mu"] - it["v"].sum()
    assert math.isclose(B, want, rel_tol=1e-10, abs_tol=1e-10 * n * it["mu"])


def test_v_norm_bound_lemma42():
    """P9: ||v|| <= sqrt(3 n mu) ||f^(t)|| (Lemma 4.2; w.h.p. -- checked on fixed seeds)."""
    for seed in range(3):
        it = _one_iteration(seed=seed)
        f = math.sqrt(max(it["sol"]["cg"].rho[-1], 0))
        n = it["x"].size
        assert np.linalg.norm(it["v"]) <= math.sqrt(3 * n * it["mu"]) * f


def _alpha_max_brute(x, s, dx, ds, gamma, eta, mu0, grid=20001):
    n = x.size
    alphas = np.linspace(0, 1, grid)
    ok_prev = 0.0
    for a in alphas:
        xn, sn = x + a * dx, s + a * ds
        mu = xn @ sn / n
        if np.any(xn * sn < (1 - gamma) * mu - 1e-15) or (1 - a) * eta > mu / mu0 + 1e-15:
            return ok_prev
        ok_prev = a
    return 1.0


def test_step_length_against_brute_force():
    """P8: alpha_max from the quadratic roots equals a fine-grid scan of N(gamma)."""
    rng = np.random.default_rng(4)
    for trial in range(30):
        n = 12
        x = rng.uniform(0.2, 2, n)
        s = rng.uniform(0.2, 2, n)
        dx = rng.standard_normal(n) * rng.uniform(0.5, 3)
        ds = rng.standard_normal(n) * rng.uniform(0.5, 3)
        gamma = rng.uniform(0.3, 0.99)
        xs = x * s
        gamma = max(gamma, 1.0 - xs.min() / xs.mean() + 0.01)   # start inside N(gamma)
        mu0 = (x @ s / n) * rng.uniform(1, 3)
        eta = rng.uniform(0, (x @ s / n) / mu0)
        amax, alpha, B, C = iipm.step_length(x, s, dx, ds, gamma, eta, mu0)
        brute = _alpha_max_brute(x, s, dx, ds, gamma, eta, mu0)
        assert abs(amax - brute) <= 1.0 / 20000 + 1e-12
        # alpha minimises mu on [0, amax]
        grid = np.linspace(0, amax, 2001)
        mus = [(x + a * dx) @ (s + a * ds) for a in grid]
        mu_a = (x + alpha * dx) @ (s + alpha * ds)
        assert mu_a <= min(mus) + 1e-12 * abs(min(mus)) + 1e-14


def test_first_crossing_cases():
    fc = iipm._first_crossing
    assert fc(1.0, -2.0, 0.0) == 0.5                  # linear
    assert fc(1.0, 1.0, 0.0) == np.inf                # increasing
    assert math.isclose(float(fc(2.0, -3.0, 1.0)), 1.0)  # roots 1 and 2 -> first is 1
    assert fc(1.0, 0.0, 1.0) == np.inf                # no real root
    assert math.isclose(float(fc(1.0, 0.0, -4.0)), 0.5)  # concave, root 0.5
    assert fc(0.0, 1.0, -0.5) == 2.0                  # starts on 0, leaves at 2


# ------------------------------------------------------------------ planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """A dropped term, a wrong sign and a transposed operand in the oracle each break a pin."""
    it = _one_iteration()
    A, x, sv, rd, mu = it["A"], it["x"], it["s"], it["rd"], it["mu"]
    dy, Wu, rtil = it["sol"]["dy"], it["sol"]["Wu"], it["sol"]["rtil"]

    def bad_dropped_v(A, x, s, rd, mu, sigma, dy, Wu):
        d2 = x / s
        ds = -rd - A.T @ dy
        v = np.sqrt(x * s) * Wu
        return -x + sigma * mu / s - d2 * ds, ds, v     # S^{-1} v term dropped

    def bad_sign(A, x, s, rd, mu, sigma, dy, Wu):
        d2 = x / s
        ds = -rd + A.T @ dy                               # sign flipped
        v = np.sqrt(x * s) * Wu
        return -x + sigma * mu / s - d2 * ds - v / s, ds, v

    for bad in (bad_dropped_v, bad_sign):
        dx, ds, v = bad(A, x, sv, rd, mu, 0.5, dy, Wu)
        ok_p = np.allclose(A @ dx, -it["rp"], atol=1e-9 * np.abs(it["rp"]).max())
        ok_d = np.allclose(A.T @ dy + ds, -rd, atol=1e-12)
        assert not (ok_p and ok_d)
    # transposed sketch operand: u = (A D W) q instead of (A D W)^T q is caught by Eq. addl
    G, qhat = it["sol"]["G"], it["sol"]["qhat"]
    with pytest.raises(ValueError):
        G @ qhat  # shape mismatch already; pad to square to make the mistake silent
    Gs = G[:, : G.shape[0]]
    u_bad = np.zeros(G.shape[1])
    u_bad[: G.shape[0]] = Gs @ qhat
    Wu_bad = iipm.apply_W(u_bad, it["sol"]["bucket"], it["sol"]["sign"])
    v_bad = np.sqrt(x * sv) * Wu_bad
    assert np.linalg.norm(A @ (v_bad / sv) - rtil) > 1e-3 * np.linalg.norm(rtil)


def test_l1svm_lp_matches_highs_and_separates():
    """The l1-SVM LP (App. D.1 formulation on synthetic separable data, Table 1's problem class):
    the oracle's optimum equals HiGHS's, and the (w, b) it returns separates the training points
    with margin 1 up to the tolerance."""
    from scipy.optimize import linprog

    pts, feats = 20, 200
    lp = synth.l1svm_lp(0, pts, feats)
    A = lp.A.astype(np.float64)
    hi = linprog(lp.c, A_eq=A, b_eq=lp.b, bounds=(0, None), method="highs")
    assert hi.status == 0
    for variant in ("sketch", "exact"):
        r = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(), variant=variant)
        assert r.converged and r.kkt <= 1e-8
        assert abs(r.obj - hi.fun) <= 1e-6 * abs(hi.fun)
    w = r.x[:feats] - r.x[feats:2 * feats]
    b = r.x[2 * feats] - r.x[2 * feats + 1]
    YX = A[:, :feats]                       # rows y_i x_i^T
    y = A[:, 2 * feats]                     # labels
    margins = YX @ w + y * b
    assert margins.min() >= 1 - 1e-6


def test_ipm_with_gaussian_sketch_matches_highs():
    """Algorithm 2 with the Gaussian sketch (Sec. 5, the paper's experiments) on the m=40,
    n=2000 LP: HiGHS's optimum, iterations within one of the exact-direction variant."""
    from scipy.optimize import linprog

    lp = synth.dense_lp(0, 40, 2000)
    A = lp.A.astype(np.float64)
    hi = linprog(lp.c, A_eq=A, b_eq=lp.b, bounds=(0, None), method="highs")
    ex = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(), variant="exact")
    g = iipm.ipm_solve(A, lp.b, lp.c, iipm.Params(sketch_kind="gaussian"))
    assert g.converged and g.kkt <= 1e-8
    assert abs(g.obj - hi.fun) <= 1e-6 * abs(hi.fun)
    assert abs(g.iters - ex.iters) <= 1
