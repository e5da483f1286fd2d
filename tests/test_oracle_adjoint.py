"""Pins of the implicit-differentiation oracle."""
import numpy as np
import pytest

from instances import tiny_lp, random_block_lp
from oracle import adjoint, ipm, lp as lpm
from helpers import load_golden


def test_closed_form_textbook():
    """Nondegenerate optimum: dObj/dc = x*, dObj/db = y* (LP sensitivity)."""
    lp, d = load_golden("lp_textbook_2x4.json")
    A, b, c = lpm.assemble(lp)
    r = ipm.solve(A, b, c, tol=1e-12)
    gc, gb = adjoint.objective_gradients(A, c, r["x"], r["z"])
    np.testing.assert_allclose(gc, d["x"], atol=1e-6)
    np.testing.assert_allclose(gb, d["y"], atol=1e-6)


@pytest.mark.parametrize("seed", [1, 2])
def test_closed_form_planted_nondegenerate(seed):
    lp = random_block_lp(seed, N=2, m_sizes=[3, 3], n_sizes=[6, 6], nnz_per_col=2, n0=1,
                         w_density=1.0, l=1, link_nnz=(2, 2), plant="nondegenerate")
    A, b, c = lpm.assemble(lp)
    r = ipm.solve(A, b, c, tol=1e-12)
    gc, gb = adjoint.objective_gradients(A, c, r["x"], r["z"])
    np.testing.assert_allclose(gc, lp.xstar, atol=1e-6)
    np.testing.assert_allclose(gb, lp.ystar, atol=1e-6)


def test_central_differences():
    lp = random_block_lp(3, N=2, m_sizes=[3, 3], n_sizes=[6, 6], nnz_per_col=2, n0=1,
                         w_density=1.0, l=1, link_nnz=(2, 2), plant="nondegenerate")
    A, b, c = lpm.assemble(lp)
    r = ipm.solve(A, b, c, tol=1e-12)
    gc, gb = adjoint.objective_gradients(A, c, r["x"], r["z"])
    h = 1e-6
    rng = np.random.default_rng(0)
    for k in rng.choice(len(c), 4, replace=False):
        e = np.zeros(len(c)); e[k] = h
        fp = ipm.solve(A, b, c + e, tol=1e-12)["pobj"]
        fm = ipm.solve(A, b, c - e, tol=1e-12)["pobj"]
        assert abs((fp - fm) / (2 * h) - gc[k]) <= 1e-5 * (1 + abs(gc[k]))
    for k in rng.choice(len(b), 3, replace=False):
        e = np.zeros(len(b)); e[k] = h
        fp = ipm.solve(A, b + e, c, tol=1e-12)["pobj"]
        fm = ipm.solve(A, b - e, c, tol=1e-12)["pobj"]
        assert abs((fp - fm) / (2 * h) - gb[k]) <= 1e-5 * (1 + abs(gb[k]))


def test_vjp_x_matches_fd():
    lp = random_block_lp(4, N=2, m_sizes=[3, 3], n_sizes=[6, 6], nnz_per_col=2, n0=1,
                         w_density=1.0, l=1, link_nnz=(2, 2), plant="nondegenerate")
    A, b, c = lpm.assemble(lp)
    r = ipm.solve(A, b, c, tol=1e-12)
    rng = np.random.default_rng(1)
    g = rng.standard_normal(len(c))
    lx, ly = adjoint.vjp_x(A, r["x"], r["z"], g)
    # at a nondegenerate vertex x* is locally constant in c and affine in b
    assert np.abs(lx).max() < 1e-5
    h = 1e-6
    k = 0
    e = np.zeros(len(b)); e[k] = h
    xp = ipm.solve(A, b + e, c, tol=1e-12)["x"]
    xm = ipm.solve(A, b - e, c, tol=1e-12)["x"]
    assert abs(g @ (xp - xm) / (2 * h) - ly[k]) <= 1e-5 * (1 + abs(ly[k]))
