"""Brute-force vertex enumeration for tiny standard-form LPs.

A bounded feasible LP min c'x, Ax = b, x >= 0 with A of full row rank attains
its optimum at a basic feasible solution (fundamental theorem of LP).  Trying
every column subset B of size m with A_B nonsingular and x_B = A_B^-1 b >= 0
therefore finds the optimal objective.  Exponential; for m <= 8, n <= 16.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np


def enumerate_optimum(A, b, c, feas_tol: float = 1e-9):
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A, dtype=float)
    m, n = A.shape
    if np.linalg.matrix_rank(A) < m:
        raise ValueError("A must have full row rank")
    best, best_x, count = np.inf, None, 0
    for B in combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-12:
            continue
        xB = np.linalg.solve(AB, b)
        if np.min(xB) < -feas_tol:
            continue
        count += 1
        x = np.zeros(n)
        x[list(B)] = xB
        val = float(c @ x)
        if val < best:
            best, best_x = val, x
    return best, best_x, count
