"""Brute-force vertex enumeration for tiny standard-form LPs.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A bounded feasible LP min c^T x, A x = b, x >= 0 with rank(A) = m attains its
optimum at a basic feasible solution: choose m columns B with A_B
nonsingular, set x_B = A_B^{-1} b, x_N = 0, keep it if x_B >= 0.  Trying all
C(n, m) bases gives the exact optimum (fundamental theorem of LP).
"""
from __future__ import annotations

import itertools

import numpy as np


def vertex_optimum(A, b, c, feas_tol: float = 1e-10):
    """Returns (best objective, best x) over all basic feasible solutions."""
    m, n = A.shape
    best, best_x = np.inf, None
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-12:
            continue
        xB = np.linalg.solve(AB, b)
        if np.min(xB) < -feas_tol:
            continue
        x = np.zeros(n)
        x[list(B)] = xB
        obj = float(c @ x)
        if obj < best:
            best, best_x = obj, x
    return best, best_x
