"""FP64 oracle of Algorithm 2 (infeasible IPM) with Algorithm 1 (sketch-PCG).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Plain numpy/scipy in float64.  Library routines (matmul, QR, Cholesky,
triangular solve) serve as single steps; nothing is blocked, fused or
reordered beyond what the cited passage states.  ``A`` is an (m, n) float64
array or a scipy.sparse matrix; vectors are float64.

Readings of passages the paper leaves open:
  * r_p lives in R^m and r_d in R^n (Sec. 1 swaps the dimensions).
  * Q^{-1/2} is used through any factor R with R^T R = Q (Alg. 1, step 2):
    PCG with preconditioner M = Q produces the same dy iterates as CG on
    Eq. precond_alt with dy = Q^{-1/2} z.
  * CG stops when sqrt(rho_j) <= min(cg_tol * sqrt(rho_0), gamma sigma
    sqrt(mu)/(4 sqrt(n))), rho_j = ||f^(j)||^2, or after cg_max_iter steps:
    the experiments use a relative tolCG (Sec. 6); the absolute bound is the
    one Sec. 4 needs for ||v|| <= gamma sigma mu / 4 (Lemma conouter).
  * W has s nonzeros per row (default s = 4; s = 1 is CountSketch), w = 4m.
  * alpha_max keeps the whole segment [0, alpha] inside N(gamma)
    (Lemma 3.5 of App. C); residuals move as r(alpha) = (1 - alpha) r.
  * step (f) minimises mu(alpha) on [0, alpha_max]; ties take the larger alpha.
  * the loop stops on scaled primal, dual and gap residuals all <= tol.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np
import scipy.linalg as sla

from .hashing import gaussian_W, sketch_indices


@dataclasses.dataclass
class Params:
    tol: float = 1e-8
    sigma: float = 0.5          # centering parameter, Sec. 6 default; must be < 4/5 (Alg. 2)
    gamma: float = 0.99         # N(gamma) width; not stated for the experiments
    cg_tol: float = 1e-6
    cg_max_iter: int = 500
    ipm_max_iter: int = 200
    sketch_s: int = 4           # nonzeros per row of W (1 = CountSketch; 4 = sparse sign)
    sketch_w: int = 0           # 0 -> 4 m
    seed: int = 0
    refine_max: int = 6         # steps of the FP64 refinement of Q^{-1} r~ (Sec. 4, Eq. compv)
    cg_theory_rule: bool = True # also stop only once ||f|| <= gamma sigma sqrt(mu)/(4 sqrt(n)) (Sec. 4)
    inner: str = "cg"           # "cg" (Alg. 1 step 3) or "richardson" (App. A)
    sketch_kind: str = "sparse" # "sparse" (s nonzeros per row) or "gaussian" (Sec. 5, Sec. 6)


# --------------------------------------------------------------------------
# Alg. 2 step (b): residuals, duality measure and right-hand side
# --------------------------------------------------------------------------

def residuals(A, b, c, x, y, s):
    """r_p = A x - b, r_d = A^T y + s - c, mu = x^T s / n (Sec. 4, Eq. update)."""
    n = x.shape[0]
    rp = A @ x - b
    rd = A.T @ y + s - c
    mu = float(x @ s) / n
    return rp, rd, mu


def rhs_p(A, b, x, s, rp, rd, mu, sigma):
    """p of Eq. pdef: p = -r_p - sigma mu A S^{-1} 1 + A x - A D^2 r_d.

    Written out literally, term by term, with D^2 = X S^{-1} (Sec. 1).
    """
    d2 = x / s
    return -rp - sigma * mu * (A @ (1.0 / s)) + A @ x - A @ (d2 * rd)


def rhs_p_short(A, b, x, s, rd, mu, sigma):
    """The same p simplified with r_p = A x - b: p = b - A(sigma mu / s + d^2 r_d)."""
    d2 = x / s
    return b - A @ (sigma * mu / s + d2 * rd)


def normal_matvec(A, d2, v):
    """A D^2 A^T v (the operator of Eq. normal)."""
    return A @ (d2 * (A.T @ v))


# --------------------------------------------------------------------------
# Alg. 1 step 1 / Alg. 2 step (a): the sketch A D W
# --------------------------------------------------------------------------

def sketch_ADW_given_W(A, d, W):
    """A D W for an explicit dense W (e.g. the Gaussian sketch of Sec. 5)."""
    return np.asarray(A @ (d[:, None] * W))


def sketch_W_dense(bucket, sign, w):
    """W as a dense (n, w) matrix (small n only): W[i, bucket[i, j]] = sign / sqrt(s)."""
    n, s = bucket.shape
    W = np.zeros((n, w))
    rows = np.repeat(np.arange(n), s)
    np.add.at(W, (rows, bucket.reshape(-1)), sign.reshape(-1) / math.sqrt(s))
    return W


def sketch_ADW(A, d, bucket, sign, w):
    """A D W (m x w, Eq. pdprecond) by scatter-adding the scaled columns of A.

    Column i of A D contributes sign(i, j)/sqrt(s) * d_i * A[:, i] to column
    bucket(i, j) of the sketch, for each of its s nonzeros j.
    """
    n, s = bucket.shape
    m = A.shape[0]
    G = np.zeros((w, m))  # rows of (A D W)^T
    scale = 1.0 / math.sqrt(s)
    if hasattr(A, "tocsc"):
        ADt = (A.multiply(d[None, :])).T.tocsr()  # n x m, row i = d_i A[:, i]^T
        for j in range(s):
            coef = sign[:, j] * scale
            import scipy.sparse as sp
            P = sp.csr_matrix((coef, (bucket[:, j], np.arange(n))), shape=(w, n))
            G += (P @ ADt).toarray()
    else:
        ADt = (A * d[None, :]).T  # n x m
        for j in range(s):
            np.add.at(G, bucket[:, j], (sign[:, j] * scale)[:, None] * ADt)
    return np.ascontiguousarray(G.T)


def apply_W(u, bucket, sign):
    """(W u)_i = sum_j sign(i, j)/sqrt(s) * u[bucket(i, j)]  (a gather per row of W)."""
    s = bucket.shape[1]
    return (sign * u[bucket]).sum(axis=1) / math.sqrt(s)


# --------------------------------------------------------------------------
# Alg. 1 step 2: factor of Q = (A D W)(A D W)^T
# --------------------------------------------------------------------------

def factor_R(G):
    """Upper-triangular R (m x m) with R^T R = G G^T = Q, from a QR of G^T.

    Alg. 1 uses the SVD of A D W to build Q^{-1/2}; any R with R^T R = Q yields
    the same preconditioned CG iterates, and QR avoids squaring the condition
    number.  Raises numpy.linalg.LinAlgError if A D W is rank deficient
    (Lemma 4.1 gives full rank only with high probability).
    """
    R = np.linalg.qr(G.T, mode="r")
    dg = np.abs(np.diag(R))
    if dg.size and (dg.min() <= 1e-14 * dg.max()):
        raise np.linalg.LinAlgError("A D W is rank deficient")
    return R


def q_inverse_apply(R, r):
    """Q^{-1} r = R^{-1} R^{-T} r through two triangular solves."""
    t = sla.solve_triangular(R, r, trans="T", lower=False)
    return sla.solve_triangular(R, t, lower=False)


def q_inv_half_svd(G):
    """Q^{-1/2} = U_Q Sigma_Q^{-1/2} U_Q^T from the SVD of A D W (Alg. 1, steps 1-2).

    Alg. 1 calls the singular values of A D W "Sigma_Q^{1/2}"; with
    singular values sigma_i the inverse square root of Q has eigenvalues
    1/sigma_i.
    """
    U, sv, _ = np.linalg.svd(G, full_matrices=False)
    return (U / sv[None, :]) @ U.T


# --------------------------------------------------------------------------
# Alg. 1 step 3: CG on the preconditioned system
# --------------------------------------------------------------------------

@dataclasses.dataclass
class CGResult:
    dy: np.ndarray
    iters: int
    rho: list            # rho_j = r_j^T Q^{-1} r_j = ||f^(j)||^2, j = 0..iters
    converged: bool


def pcg(matvec: Callable, p, prec: Callable, tol: float, max_iter: int,
        abs_tol: float = math.inf) -> CGResult:
    """Preconditioned CG for (A D^2 A^T) dy = p with preconditioner Q (Alg. 1 step 3).

    Starts from dy = 0 (z^0 = 0).  ``prec(r)`` applies Q^{-1}.  rho_j equals
    the squared norm of the residual f^(j) of Eq. precond_alt (Sec. 3), and
    the loop stops once sqrt(rho_j) <= min(tol * sqrt(rho_0), abs_tol) or
    after max_iter products with A D^2 A^T.
    """
    dy = np.zeros_like(p)
    r = p.copy()
    z = prec(r)
    d = z.copy()
    rho = float(r @ z)
    hist = [rho]
    thresh = min(tol * math.sqrt(rho), abs_tol) if rho > 0 else 0.0
    it = 0
    converged = rho <= 0
    while not converged and it < max_iter:
        q = matvec(d)
        dq = float(d @ q)
        alpha = rho / dq
        dy += alpha * d
        r -= alpha * q
        z = prec(r)
        rho_new = float(r @ z)
        it += 1
        hist.append(rho_new)
        if math.sqrt(max(rho_new, 0.0)) <= thresh:
            converged = True
            break
        beta = rho_new / rho
        d = z + beta * d
        rho = rho_new
    return CGResult(dy=dy, iters=it, rho=hist, converged=converged)


def cg_precond_alt(matvec: Callable, p, Qmh, tol: float, max_iter: int) -> CGResult:
    """Plain CG on Eq. precond_alt, Q^{-1/2} A D^2 A^T Q^{-1/2} z = Q^{-1/2} p.

    Returns dy = Q^{-1/2} z (Alg. 2 step (c)); ``rho`` holds ||f^(j)||^2.
    A second, independent route to the same iterates as ``pcg``.
    """
    rhs = Qmh @ p
    z = np.zeros_like(p)
    r = rhs.copy()
    d = r.copy()
    rho = float(r @ r)
    hist = [rho]
    thresh = tol * math.sqrt(rho)
    it = 0
    converged = rho <= 0
    while not converged and it < max_iter:
        q = Qmh @ matvec(Qmh @ d)
        alpha = rho / float(d @ q)
        z += alpha * d
        r -= alpha * q
        rho_new = float(r @ r)
        it += 1
        hist.append(rho_new)
        if math.sqrt(rho_new) <= thresh:
            converged = True
            break
        d = r + (rho_new / rho) * d
        rho = rho_new
    return CGResult(dy=Qmh @ z, iters=it, rho=hist, converged=converged)


def richardson(matvec: Callable, p, Qmh, max_iter: int, tol: float = 0.0,
               abs_tol: float = math.inf) -> CGResult:
    """Richardson's iteration of App. A in place of Alg. 1 step 3.

    z^0 = 0 and z^j = z^{j-1} + Q^{-1/2} (p - A D^2 A^T Q^{-1/2} z^{j-1}); the
    output is dy = Q^{-1/2} z^t.  ``rho`` holds ||f~^(j)||^2 with
    f~^(j) = Q^{-1/2} (A D^2 A^T Q^{-1/2} z^j - p), the residual of Lemma
    recursive.  App. A runs a fixed number t of steps; here it also stops, like
    CG, once ||f~^(j)|| <= min(tol ||f~^(0)||, abs_tol) (tol = 0: exactly
    max_iter steps).  ``Qmh`` is Q^{-1/2}.
    """
    z = np.zeros_like(p)
    f = -(Qmh @ p)                      # f~^(0) = -Q^{-1/2} p
    rho = float(f @ f)
    hist = [rho]
    thresh = min(tol * math.sqrt(rho), abs_tol)
    it = 0
    converged = False
    while it < max_iter:
        z = z + Qmh @ (p - matvec(Qmh @ z))
        f = Qmh @ (matvec(Qmh @ z) - p)
        it += 1
        hist.append(float(f @ f))
        if math.sqrt(hist[-1]) <= thresh:
            converged = True
            break
    return CGResult(dy=Qmh @ z, iters=it, rho=hist, converged=converged)


# --------------------------------------------------------------------------
# Alg. 2 step (d): correction vector v and the corrected direction
# --------------------------------------------------------------------------

def correction_u(G, R, rtil, refine_max: int):
    """u = (A D W)^dagger r~ = (A D W)^T Q^{-1} r~ (Eq. compv; full row rank, Lemma 4.1).

    Q^{-1} r~ is taken through R and refined in FP64 against Q = G G^T
    until the correction stops shrinking.  Returns (u, qhat, steps).
    """
    qhat = q_inverse_apply(R, rtil)
    prev = math.inf
    steps = 0
    for _ in range(refine_max):
        res = rtil - G @ (G.T @ qhat)
        nr = float(np.linalg.norm(res))
        if nr >= 0.5 * prev or nr == 0.0:
            break
        qhat = qhat + q_inverse_apply(R, res)
        prev = nr
        steps += 1
    return G.T @ qhat, qhat, steps


def directions(A, x, s, rd, mu, sigma, dy, Wu):
    """Corrected directions of Sec. 4.

    ds = -r_d - A^T dy                       (Eq. delshat)
    v  = (X S)^{1/2} W u                     (Eq. compv, with u = (A D W)^dagger r~)
    dx = -x + sigma mu S^{-1} 1 - D^2 ds - S^{-1} v   (Eq. delxhat)
    """
    d2 = x / s
    ds = -rd - A.T @ dy
    v = np.sqrt(x * s) * Wu
    dx = -x + sigma * mu / s - d2 * ds - v / s
    return dx, ds, v


# --------------------------------------------------------------------------
# Alg. 2 steps (e)-(f): step length
# --------------------------------------------------------------------------

def _first_crossing(a0, a1, a2):
    """Smallest alpha in (0, 1] where a0 + a1 a + a2 a^2 turns negative (inf if none).

    Elementwise over arrays.  Roots come from the cancellation-free quadratic
    formula q = -(a1 + sign(a1) sqrt(disc))/2, roots q/a2 and a0/q; a root
    counts only where the polynomial's slope is negative.
    """
    a0 = np.maximum(np.asarray(a0, dtype=np.float64), 0.0)
    a1 = np.asarray(a1, dtype=np.float64)
    a2 = np.asarray(a2, dtype=np.float64)
    a0, a1, a2 = np.broadcast_arrays(a0, a1, a2)
    out = np.full(a0.shape, np.inf)
    with np.errstate(divide="ignore", invalid="ignore"):
        lin = a2 == 0.0
        # linear case
        r_lin = np.where(a1 < 0, a0 / (-a1), np.inf)
        out = np.where(lin, r_lin, out)
        disc = a1 * a1 - 4.0 * a2 * a0
        ok = (~lin) & (disc >= 0)
        sq = np.sqrt(np.where(ok, disc, 0.0))
        qq = -0.5 * (a1 + np.where(a1 >= 0, sq, -sq))
        r1 = np.where(ok & (a2 != 0), qq / a2, np.inf)
        r2 = np.where(ok & (qq != 0), a0 / qq, np.inf)
        best = np.full(a0.shape, np.inf)
        for r in (r1, r2):
            slope = 2.0 * a2 * r + a1
            good = ok & np.isfinite(r) & (r > 0) & (slope < 0)
            best = np.where(good & (r < best), r, best)
        out = np.where(lin, out, best)
    return out


def step_length(x, s, dx, ds, gamma, eta, mu0):
    """alpha_max and alpha of Alg. 2 steps (e) and (f).

    N(gamma) (Sec. 4): x_i s_i >= (1 - gamma) mu and ||r||/||r^0|| <= mu/mu_0.
    mu(a) = (x^T s + a B + a^2 C)/n with B = x^T ds + s^T dx, C = dx^T ds.
    Each condition along the segment is a quadratic in a:
      q_i(a) = (x_i + a dx_i)(s_i + a ds_i) - (1 - gamma) mu(a) >= 0,
      g(a)   = mu(a)/mu_0 - (1 - a) eta >= 0,   eta = ||r||/||r^0||,
    using r(a) = (1 - a) r, which Eq. addl guarantees (App. C, Eq. iip_3).
    alpha_max is the first crossing in (0, 1], else 1.  alpha minimises mu(a)
    on [0, alpha_max] (ties -> larger a).  Returns (alpha_max, alpha, B, C).
    """
    n = x.shape[0]
    xs = float(x @ s)
    B = float(x @ ds + s @ dx)
    C = float(dx @ ds)
    g1 = 1.0 - gamma
    a0 = x * s - g1 * xs / n
    a1 = x * ds + s * dx - g1 * B / n
    a2 = dx * ds - g1 * C / n
    amax = min(1.0, float(np.min(_first_crossing(a0, a1, a2))) if n else 1.0)
    g = _first_crossing(xs / n / mu0 - eta, B / n / mu0 + eta, C / n / mu0)
    amax = min(amax, float(g))
    # step (f): minimise B a + C a^2 on [0, amax]
    cand = [0.0, amax]
    if C > 0:
        v = -B / (2.0 * C)
        if 0.0 < v < amax:
            cand.append(v)
    f = lambda a: B * a + C * a * a
    best = max(cand, key=lambda a: (-f(a), a))
    return amax, best, B, C


# --------------------------------------------------------------------------
# Alg. 2: the outer loop
# --------------------------------------------------------------------------

@dataclasses.dataclass
class IterLog:
    k: int
    mu: float
    rp_rel: float
    rd_rel: float
    gap_rel: float
    cg_iters: int
    alpha_max: float
    alpha: float
    v_norm: float
    f_norm: float


@dataclasses.dataclass
class IPMResult:
    x: np.ndarray
    y: np.ndarray
    s: np.ndarray
    iters: int
    converged: bool
    obj: float
    kkt: float
    cg_total: int
    log: list


def kkt_scaled(A, b, c, x, y, s):
    """max of ||r_p||/(1+||b||), ||r_d||/(1+||c||), n mu/(1+|c^T x|) (stopping rule)."""
    rp, rd, mu = residuals(A, b, c, x, y, s)
    n = x.shape[0]
    return (float(np.linalg.norm(rp)) / (1 + float(np.linalg.norm(b))),
            float(np.linalg.norm(rd)) / (1 + float(np.linalg.norm(c))),
            n * mu / (1 + abs(float(c @ x))))


def cg_abs_threshold(x, s, prm: Params):
    """gamma sigma sqrt(mu) / (4 sqrt(n)): the bound on ||f^(t)|| that makes
    ||v|| <= gamma sigma mu / 4 (Sec. 4 after Lemma 4.2; Lemma conouter, App. C)."""
    if not prm.cg_theory_rule:
        return math.inf
    n = x.shape[0]
    mu = float(x @ s) / n
    return prm.gamma * prm.sigma * math.sqrt(mu) / (4.0 * math.sqrt(n))


def normal_solve_sketch(A, x, s, p, k, prm: Params):
    """Alg. 1 plus the correction of Eq. compv for one iterate (x, s) and RHS p.

    Returns a dict with dy, cg result, G = A D W, R, r~ = A D^2 A^T dy - p,
    u, Wu, bucket and sign.
    """
    m, n = A.shape
    w = prm.sketch_w or 4 * m
    d2 = x / s
    d = np.sqrt(d2)
    if prm.sketch_kind == "gaussian":
        Wg = gaussian_W(prm.seed, k, n, w)
        G = sketch_ADW_given_W(A, d, Wg)
        bucket = sign = None
    else:
        bucket, sign = sketch_indices(prm.seed, k, n, prm.sketch_s, w)
        G = sketch_ADW(A, d, bucket, sign, w)
    R = factor_R(G)
    mv = lambda v: normal_matvec(A, d2, v)
    if prm.inner == "richardson":
        cg = richardson(mv, p, q_inv_half_svd(G), prm.cg_max_iter, prm.cg_tol,
                        abs_tol=cg_abs_threshold(x, s, prm))
    else:
        cg = pcg(mv, p, lambda r: q_inverse_apply(R, r), prm.cg_tol, prm.cg_max_iter,
                 abs_tol=cg_abs_threshold(x, s, prm))
    rtil = mv(cg.dy) - p
    u, qhat, steps = correction_u(G, R, rtil, prm.refine_max)
    Wu = Wg @ u if prm.sketch_kind == "gaussian" else apply_W(u, bucket, sign)
    return dict(dy=cg.dy, cg=cg, G=G, R=R, rtil=rtil, u=u, Wu=Wu, qhat=qhat,
                refine_steps=steps, bucket=bucket, sign=sign, w=w)


def ipm_solve(A, b, c, prm: Optional[Params] = None, variant: str = "sketch",
              start=None, callback=None) -> IPMResult:
    """Algorithm 2 (infeasible long-step IPM) in FP64.

    variant "sketch": Alg. 1 (sketch-preconditioned CG) plus the correction
    vector v of Eq. compv.  variant "exact": dy from a Cholesky factor of
    A D^2 A^T and v = 0 (the "IPM w/ Dir." comparator of Sec. 6).
    Start (x, y, s) = (1, 0, 1) unless ``start`` is given.
    """
    prm = prm or Params()
    m, n = A.shape
    if start is None:
        x, y, s = np.ones(n), np.zeros(m), np.ones(n)
    else:
        x, y, s = (np.array(t, dtype=np.float64) for t in start)
    rp0, rd0, mu0 = residuals(A, b, c, x, y, s)
    r0 = math.sqrt(float(rp0 @ rp0 + rd0 @ rd0))
    log = []
    cg_total = 0
    k = 0
    converged = False
    while True:
        rp, rd, mu = residuals(A, b, c, x, y, s)
        e_p, e_d, e_g = kkt_scaled(A, b, c, x, y, s)
        if max(e_p, e_d, e_g) <= prm.tol:
            converged = True
            break
        if k >= prm.ipm_max_iter:
            break
        d2 = x / s
        p = rhs_p(A, b, x, s, rp, rd, mu, prm.sigma)
        if variant == "exact":
            K = (A @ (d2[:, None] * A.T.toarray() if hasattr(A, "tocsc") else d2[:, None] * A.T))
            K = np.asarray(K)
            cf = sla.cho_factor(K)
            dy = sla.cho_solve(cf, p)
            Wu = np.zeros(n)
            cg_it, fnorm = 0, 0.0
        else:
            sol = normal_solve_sketch(A, x, s, p, k, prm)
            dy, Wu = sol["dy"], sol["Wu"]
            cg_it = sol["cg"].iters
            fnorm = math.sqrt(max(sol["cg"].rho[-1], 0.0))
        cg_total += cg_it
        dx, ds, v = directions(A, x, s, rd, mu, prm.sigma, dy, Wu)
        eta = math.sqrt(float(rp @ rp + rd @ rd)) / r0 if r0 > 0 else 0.0
        amax, alpha, _, _ = step_length(x, s, dx, ds, prm.gamma, eta, mu0)
        log.append(IterLog(k=k, mu=mu, rp_rel=e_p, rd_rel=e_d, gap_rel=e_g, cg_iters=cg_it,
                           alpha_max=amax, alpha=alpha, v_norm=float(np.linalg.norm(v)),
                           f_norm=fnorm))
        if callback is not None:
            callback(k, locals())
        x = x + alpha * dx
        y = y + alpha * dy
        s = s + alpha * ds
        k += 1
    e = kkt_scaled(A, b, c, x, y, s)
    return IPMResult(x=x, y=y, s=s, iters=k, converged=converged, obj=float(c @ x),
                     kkt=max(e), cg_total=cg_total, log=log)
