"""The primal-dual Newton system, solved monolithically.

Sec. 2.3: at an interior point (x, z > 0) the Newton step solves

    [ 0  A'  I ] [dx]   [r_d]
    [ A  0   0 ] [dy] = [r_p]
    [ Z  0   X ] [dz]   [r_c]

Eliminating dz = X^-1 (r_c - Z dx) gives the augmented system (eq.
linear_system_aug_ipm)

    [ -X^-1 Z  A' ] [dx]   [ r_d - X^-1 r_c ]
    [   A      0  ] [dy] = [      r_p       ]

``direction_dense`` solves the 3x3 system itself with LAPACK (plain
definition); ``direction_sparse`` factors the augmented system with SuperLU
and back-substitutes dz.  No block structure is used anywhere here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def newton_matrix_dense(A, x, z) -> np.ndarray:
    A = A.toarray() if sp.issparse(A) else np.asarray(A)
    m, n = A.shape
    J = np.zeros((2 * n + m, 2 * n + m))
    J[:n, n:n + m] = A.T
    J[:n, n + m:] = np.eye(n)
    J[n:n + m, :n] = A
    J[n + m:, :n] = np.diag(z)
    J[n + m:, n + m:] = np.diag(x)
    return J


def direction_dense(A, x, z, r_d, r_p, r_c):
    """Solve the 3x3 Newton system with LU (numpy.linalg.solve)."""
    m, n = A.shape
    J = newton_matrix_dense(A, x, z)
    d = np.linalg.solve(J, np.concatenate([r_d, r_p, r_c]))
    return d[:n], d[n:n + m], d[n + m:]


def augmented_matrix(A, x, z):
    A = sp.csr_matrix(A)
    m, n = A.shape
    return sp.bmat([[sp.diags(-z / x), A.T], [A, sp.csr_matrix((m, m))]], format="csc")


def direction_sparse(A, x, z, r_d, r_p, r_c):
    """Sparse LU of the augmented system, then dz = X^-1 (r_c - Z dx)."""
    m, n = A.shape
    K = augmented_matrix(A, x, z)
    lu = spla.splu(K)
    sol = lu.solve(np.concatenate([r_d - r_c / x, r_p]))
    dx, dy = sol[:n], sol[n:]
    dz = (r_c - z * dx) / x
    return dx, dy, dz


def direction(A, x, z, r_d, r_p, r_c, dense_limit: int = 4000):
    m, n = A.shape
    if 2 * n + m <= dense_limit:
        return direction_dense(A, x, z, r_d, r_p, r_c)
    return direction_sparse(A, x, z, r_d, r_p, r_c)


def residual(A, x, z, dx, dy, dz, r_d, r_p, r_c):
    """Blocks of J d - r by sparse mat-vecs (no factorization)."""
    return (A.T @ dy + dz - r_d, A @ dx - r_p, z * dx + x * dz - r_c)


def relative_residual(A, x, z, dx, dy, dz, r_d, r_p, r_c) -> float:
    e = np.concatenate(residual(A, x, z, dx, dy, dz, r_d, r_p, r_c))
    r = np.concatenate([r_d, r_p, r_c])
    return float(np.linalg.norm(e) / max(np.linalg.norm(r), 1e-300))
