"""Pins of the monolithic Newton direction (Sec. 2.3)."""
import numpy as np
import pytest

from instances import config0, random_block_lp
from oracle import newton, lp as lpm


def _point(lp, seed=0, spread=1.0):
    A, b, c = lpm.assemble(lp)
    rng = np.random.default_rng(seed)
    m, n = A.shape
    x = np.exp(spread * rng.standard_normal(n))
    z = np.exp(spread * rng.standard_normal(n))
    return A, b, c, x, z, rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n)


def test_dense_and_sparse_agree():
    """3x3 LAPACK solve vs SuperLU on the augmented form with dz eliminated."""
    lp = config0()
    A, b, c, x, z, rd, rp, rc = _point(lp)
    d1 = newton.direction_dense(A, x, z, rd, rp, rc)
    d2 = newton.direction_sparse(A, x, z, rd, rp, rc)
    for u, v in zip(d1, d2):
        np.testing.assert_allclose(u, v, rtol=1e-9, atol=1e-9)
    assert newton.relative_residual(A, x, z, *d1, rd, rp, rc) < 1e-12


def test_least_norm_special_case():
    """x = z = 1, r_d = r_c = 0: dx is the minimum-norm solution of A dx = r_p."""
    lp = config0(seed=3)
    A, b, c, x, z, rd, rp, rc = _point(lp)
    n = A.shape[1]
    one = np.ones(n)
    dx, dy, dz = newton.direction_dense(A, one, one, np.zeros(n), rp, np.zeros(n))
    ref = np.linalg.lstsq(A.toarray(), rp, rcond=None)[0]
    np.testing.assert_allclose(dx, ref, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(dz, -dx, atol=1e-12)


def test_full_step_restores_feasibility():
    """A(x + dx) = b when r_p = b - Ax (linearity of the primal rows)."""
    lp = config0(seed=4)
    A, b, c, x, z, rd, rp, rc = _point(lp)
    y = np.zeros(A.shape[0])
    r_p = b - A @ x
    r_d = c - A.T @ y - z
    dx, dy, dz = newton.direction(A, x, z, r_d, r_p, rc)
    np.testing.assert_allclose(A @ (x + dx), b, atol=1e-9)
    np.testing.assert_allclose(A.T @ (y + dy) + (z + dz), c, atol=1e-9)


def test_complementarity_row():
    """Z dx + X dz = r_c holds exactly up to rounding (Sec. 2.3 elimination)."""
    lp = random_block_lp(2, N=3, m_sizes=[5, 6, 4], n_sizes=[8, 9, 7], nnz_per_col=2,
                         n0=2, w_density=0.5, l=[1, 2], mg=1)
    A, b, c, x, z, rd, rp, rc = _point(lp, spread=2.0)
    dx, dy, dz = newton.direction_sparse(A, x, z, rd, rp, rc)
    np.testing.assert_allclose(z * dx + x * dz, rc, rtol=1e-10, atol=1e-10)
