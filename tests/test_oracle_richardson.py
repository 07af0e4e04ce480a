"""P11: pins of the oracle's Richardson iteration (App. A) to what the appendix proves.

Lemma recursive gives f~^(j) = (I - Q^-1/2 A D^2 A^T Q^-1/2) f~^(j-1), and Lemma normbound
bounds that matrix's norm by zeta < 1 when the sketch satisfies Eq. pdcond1; so
||f~^(t)|| <= zeta^t ||Q^-1/2 p||.  zeta is computed here through a route the iteration does
not use (the eigenvalues of V^T W W^T V, V the right singular vectors of A D, whose
reciprocals are the preconditioned spectrum, proof of Lemma 3.1).  The limit is checked against
a Cholesky solve, the dy-space form (the GPU's) against the z-space form, and a full IPM with
Richardson against SciPy HiGHS.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import hashing, iipm


def _setup(m=12, n=3000, w_mult=40, s=4, seed=5, spread=3.0):
    lp = synth.dense_lp(seed, m, n)
    A = lp.A.astype(np.float64)
    x, y, sv = synth.iterate_point(seed, m, n, spread=spread)
    d2 = x / sv
    w = w_mult * m
    b, sg = hashing.sketch_indices(0, 1, n, s, w)
    G = iipm.sketch_ADW(A, np.sqrt(d2), b, sg, w)
    W = iipm.sketch_W_dense(b, sg, w)
    _, _, Vt = np.linalg.svd(A * np.sqrt(d2)[None, :], full_matrices=False)
    ev = np.linalg.eigvalsh(Vt @ W @ W.T @ Vt.T)
    zeta = float(np.abs(1.0 - 1.0 / ev).max())   # ||I - Q^-1/2 K Q^-1/2||
    p = np.random.default_rng(seed).standard_normal(m)
    return A, d2, G, p, zeta


def test_residual_contracts_by_zeta_each_step():
    A, d2, G, p, zeta = _setup()
    assert zeta < 1
    mv = lambda v: iipm.normal_matvec(A, d2, v)
    res = iipm.richardson(mv, p, iipm.q_inv_half_svd(G), 25)
    f = np.sqrt(res.rho)
    assert res.iters == 25
    f0 = np.linalg.norm(iipm.q_inv_half_svd(G) @ p)
    assert math.isclose(f[0], f0, rel_tol=1e-12)
    # above the FP64 rounding floor (~1e-13 of f0) each step contracts by at most zeta
    live = f[:-1] > 1e-11 * f0
    assert live.sum() >= 10
    assert np.all(f[1:][live] <= zeta * f[:-1][live] * (1 + 1e-9))
    assert np.all(f <= f0 * zeta ** np.arange(len(f)) * (1 + 1e-8) + 1e-13 * f0)


def test_limit_is_the_cholesky_solution_and_dy_form_agrees():
    """Many steps reach K^-1 p; the dy-space form dy += Q^-1 (p - K dy) through the QR factor
    (the form the GPU runs) gives the same iterates as the z-space form of App. A."""
    A, d2, G, p, zeta = _setup(w_mult=60)
    K = A @ (d2[:, None] * A.T)
    dstar = sla.cho_solve(sla.cho_factor(K), p)
    mv = lambda v: iipm.normal_matvec(A, d2, v)
    t = 12
    res = iipm.richardson(mv, p, iipm.q_inv_half_svd(G), t)
    R = iipm.factor_R(G)
    dy = np.zeros_like(p)
    for _ in range(t):
        dy = dy + iipm.q_inverse_apply(R, p - mv(dy))
    assert np.linalg.norm(dy - res.dy) <= 1e-10 * np.linalg.norm(dstar)
    long = iipm.richardson(mv, p, iipm.q_inv_half_svd(G), 200)
    assert np.linalg.norm(long.dy - dstar) <= 1e-9 * np.linalg.norm(dstar)


def test_diverges_when_the_sketch_is_too_narrow():
    """With w = 4m and CountSketch the preconditioned spectrum reaches past 2: zeta > 1 and the
    residual grows (why the appendix calls Richardson impractical)."""
    A, d2, G, p, zeta = _setup(w_mult=4, s=1)
    assert zeta > 1
    mv = lambda v: iipm.normal_matvec(A, d2, v)
    res = iipm.richardson(mv, p, iipm.q_inv_half_svd(G), 60)
    assert res.rho[-1] > 100 * res.rho[0]


def test_ipm_with_richardson_matches_highs():
    """Algorithm 2 with Richardson's iteration (App. A) in place of CG, sketch w = 40m: same
    optimum as HiGHS, iterations within one of the CG variant."""
    from scipy.optimize import linprog

    lp = synth.dense_lp(2, 10, 1500)
    A = lp.A.astype(np.float64)
    hi = linprog(lp.c, A_eq=A, b_eq=lp.b, bounds=(0, None), method="highs")
    assert hi.status == 0
    prm_r = iipm.Params(inner="richardson", sketch_w=400)
    prm_c = iipm.Params(sketch_w=400)
    r = iipm.ipm_solve(A, lp.b, lp.c, prm_r)
    c = iipm.ipm_solve(A, lp.b, lp.c, prm_c)
    assert r.converged and r.kkt <= 1e-8
    assert abs(r.obj - hi.fun) <= 1e-6 * abs(hi.fun)
    assert abs(r.iters - c.iters) <= 1
    # Richardson needs more inner steps than CG for the same target
    assert r.cg_total >= c.cg_total


def test_planted_sign_mistake_is_caught():
    """A Richardson step with the correction subtracted instead of added breaks the pin."""
    A, d2, G, p, zeta = _setup()
    Qmh = iipm.q_inv_half_svd(G)
    mv = lambda v: iipm.normal_matvec(A, d2, v)
    z = np.zeros_like(p)
    f_prev = np.linalg.norm(Qmh @ p)
    ok = True
    for _ in range(5):
        z = z - Qmh @ (p - mv(Qmh @ z))
        f = np.linalg.norm(Qmh @ (mv(Qmh @ z) - p))
        ok &= f <= zeta * f_prev * (1 + 1e-9)
        f_prev = f
    assert not ok
