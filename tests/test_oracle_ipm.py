"""Pins of the oracle IPM (Sec. 2.2-2.3) against things other than itself."""
import numpy as np
import pytest

from instances import config0, tiny_lp, random_block_lp
from oracle import ipm, lp as lpm, vertex
from helpers import GOLDEN_FILES, load_golden


@pytest.mark.parametrize("name", GOLDEN_FILES)
def test_golden_hand_derived(name):
    lp, d = load_golden(name)
    A, b, c = lpm.assemble(lp)
    r = ipm.solve(A, b, c)
    assert r["status"] == "optimal"
    assert abs(r["pobj"] - d["objective"]) <= 1e-7 * (1 + abs(d["objective"]))
    np.testing.assert_allclose(r["x"], d["x"], atol=1e-6)
    if "y" in d:
        np.testing.assert_allclose(r["y"], d["y"], atol=1e-6)
        np.testing.assert_allclose(r["z"], d["z"], atol=1e-6)


@pytest.mark.parametrize("seed", range(8))
def test_vertex_enumeration(seed):
    """Brute force over all bases (fundamental theorem of LP)."""
    lp = tiny_lp(seed, N=2, m=2, n=4, n0=1, l=1, mg=1 if seed % 2 else 0)
    A, b, c = lpm.assemble(lp)
    if np.linalg.matrix_rank(A.toarray()) < A.shape[0]:
        pytest.skip("rank deficient draw")
    best, xbest, count = vertex.enumerate_optimum(A, b, c)
    assert count > 0
    r = ipm.solve(A, b, c)
    assert r["status"] == "optimal"
    assert abs(r["pobj"] - best) <= 1e-7 * (1 + abs(best))


def test_planted_optimum_c0():
    lp = config0()
    A, b, c = lpm.assemble(lp)
    r = ipm.solve(A, b, c)
    assert r["status"] == "optimal"
    obj_star = float(c @ lp.xstar)
    assert abs(obj_star - float(b @ lp.ystar)) <= 1e-12 * (1 + abs(obj_star))
    assert abs(r["pobj"] - obj_star) <= 1e-8 * (1 + abs(obj_star))
    assert r["pinf"] <= 1e-8 and r["dinf"] <= 1e-8 and r["gap"] <= 1e-8


def test_highs_crosscheck_c0():
    linprog = pytest.importorskip("scipy.optimize").linprog
    lp = config0(seed=11)
    A, b, c = lpm.assemble(lp)
    res = linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    assert res.status == 0
    r = ipm.solve(A, b, c)
    assert abs(r["pobj"] - res.fun) <= 1e-8 * (1 + abs(res.fun))


def test_measures_on_planted_point():
    """The planted point is exactly optimal: zero residuals, zero gap."""
    lp = random_block_lp(5, N=3, m_sizes=[7, 8, 6], n_sizes=[11, 12, 9], nnz_per_col=3,
                         n0=2, w_density=0.5, l=[2, 2], mg=1, x0_link_nnz=1, x0_global_nnz=1)
    A, b, c = lpm.assemble(lp)
    m = lpm.measures(A, b, c, lp.xstar, lp.ystar, lp.zstar)
    assert m["pinf"] < 1e-14 and m["dinf"] < 1e-14 and m["gap"] < 1e-14 and m["mu"] == 0.0


def test_max_step_ratio_test():
    v = np.array([1.0, 2.0, 3.0])
    assert ipm.max_step(v, np.array([-1.0, 1.0, -6.0])) == pytest.approx(0.5)
    assert ipm.max_step(v, np.array([1.0, 1.0, 0.0])) == np.inf
