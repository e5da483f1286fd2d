"""Implicit differentiation of the LP optimum through the Newton matrix.

At a solution w = (x, y, z) of F(w; c, b) = [A'y + z - c; Ax - b; XZe] = 0
the implicit function theorem gives dw = J^-1 [dc; db; 0] with J the Newton
matrix of Sec. 2.3.  For a scalar L(x) with gradient g_x (and g_y, g_z for
dependence on y, z) the vector-Jacobian product is obtained from one
transposed solve J' lam = [g_x; g_y; g_z]:  dL/dc = lam_x, dL/db = lam_y.
For the objective c'x the explicit dependence on c adds x:
dObj/dc = x + lam_x with g = [c; 0; 0], dObj/db = lam_y.
"""
from __future__ import annotations

import numpy as np

from .newton import newton_matrix_dense


def adjoint_dense(A, x, z, g_x, g_y, g_z):
    """Solve J' lam = g densely; returns (lam_x, lam_y, lam_z)."""
    m, n = A.shape
    J = newton_matrix_dense(A, x, z)
    lam = np.linalg.solve(J.T, np.concatenate([g_x, g_y, g_z]))
    return lam[:n], lam[n:n + m], lam[n + m:]


def objective_gradients(A, c, x, z):
    """(dObj/dc, dObj/db) at the point (x, z)."""
    m, n = A.shape
    lx, ly, _ = adjoint_dense(A, x, z, c, np.zeros(m), np.zeros(n))
    return x + lx, ly


def vjp_x(A, x, z, g):
    """(d(g'x)/dc, d(g'x)/db)."""
    m, n = A.shape
    lx, ly, _ = adjoint_dense(A, x, z, g, np.zeros(m), np.zeros(n))
    return lx, ly
