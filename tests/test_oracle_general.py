"""Pins of the oracle's full LP statement (Sec. 3.2: equality rows, two-sided
inequality rows, lower / upper / free / fixed bounds) against things other
than itself: hand-derived optima, and HiGHS (scipy.optimize.linprog) on
seeded random instances of every bound type."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import general

inf = np.inf


def test_hand_derived_box_free_and_inequality():
    """min -x1 - 2 x2  s.t.  x1 - x2 = 1,  x1 + x2 <= 4,  0 <= x1 <= 3, x2 free.
    With x1 = 1 + x2 the objective is -1 - 3 x2 and x1 + x2 <= 4 caps x2 at
    1.5 (x1 <= 3 would allow 2): x* = (2.5, 1.5), objective -5.5."""
    r = general.solve_general(c=[-1.0, -2.0], A=sp.csr_matrix([[1.0, -1.0]]), b=[1.0],
                              C=sp.csr_matrix([[1.0, 1.0]]), d=[-inf], f=[4.0],
                              lo=[0.0, -inf], hi=[3.0, inf])
    assert r["status"] == "optimal"
    np.testing.assert_allclose(r["x"], [2.5, 1.5], atol=1e-7)
    assert abs(r["objective"] + 5.5) <= 1e-8
    assert abs(r["standard_objective"] - r["objective"]) <= 1e-7


def test_hand_derived_upper_only_fixed_and_two_sided_row():
    """min x1 + x2 - x3  s.t.  1 <= x1 + x2 + x3 <= 2,  x1 <= 5 (no lower bound),
    x2 = 0.5 (fixed), -1 <= x3 <= 1.  Any x1 lowers the objective without
    limit unless the row binds: x1 + x3 >= 0.5 and x1 + x3 <= 1.5; with x3 = 1
    (its best value) the row leaves x1 >= -0.5, so x* = (-0.5, 0.5, 1),
    objective -1."""
    r = general.solve_general(c=[1.0, 1.0, -1.0], A=sp.csr_matrix((0, 3)), b=[],
                              C=sp.csr_matrix([[1.0, 1.0, 1.0]]), d=[1.0], f=[2.0],
                              lo=[-inf, 0.5, -1.0], hi=[5.0, 0.5, 1.0])
    assert r["status"] == "optimal"
    np.testing.assert_allclose(r["x"], [-0.5, 0.5, 1.0], atol=1e-7)
    assert abs(r["objective"] + 1.0) <= 1e-8


def _random_general(seed):
    rng = np.random.default_rng(seed)
    n, mA, mC = 9, 3, 4
    A = sp.random(mA, n, density=0.5, random_state=rng, data_rvs=rng.standard_normal).tocsr()
    C = sp.random(mC, n, density=0.5, random_state=rng, data_rvs=rng.standard_normal).tocsr()
    x0 = rng.uniform(-1, 1, n)
    kind = rng.integers(0, 4, n)   # 0 lower, 1 upper, 2 box, 3 free
    lo = np.where((kind == 0) | (kind == 2), x0 - rng.uniform(0.1, 1, n), -inf)
    hi = np.where((kind == 1) | (kind == 2), x0 + rng.uniform(0.1, 1, n), inf)
    Cx = C @ x0
    rk = rng.integers(0, 3, mC)    # 0 <=, 1 >=, 2 two-sided
    d = np.where(rk >= 1, Cx - rng.uniform(0.1, 1, mC), -inf)
    f = np.where(rk != 1, Cx + rng.uniform(0.1, 1, mC), inf)
    c = rng.standard_normal(n)
    return c, A, A @ x0, C, d, f, lo, hi


def _highs(c, A, b, C, d, f, lo, hi):
    from scipy.optimize import linprog
    Cd = C.toarray()
    rows, rhs = [], []
    for i in range(C.shape[0]):
        if np.isfinite(f[i]):
            rows.append(Cd[i])
            rhs.append(f[i])
        if np.isfinite(d[i]):
            rows.append(-Cd[i])
            rhs.append(-d[i])
    bounds = [(None if not np.isfinite(a) else a, None if not np.isfinite(z) else z)
              for a, z in zip(lo, hi)]
    return linprog(c, A_ub=np.array(rows) if rows else None, b_ub=np.array(rhs) if rows else None,
                   A_eq=A.toarray(), b_eq=b, bounds=bounds, method="highs")


def test_random_general_lps_match_highs():
    solved = 0
    for seed in range(12):
        inst = _random_general(seed)
        h = _highs(*inst)
        if h.status != 0:      # unbounded draws carry no objective to compare
            continue
        r = general.solve_general(*inst)
        assert r["status"] == "optimal", seed
        assert abs(r["objective"] - h.fun) <= 1e-7 * (1 + abs(h.fun)), (seed, r["objective"], h.fun)
        x = r["x"]
        c, A, b, C, d, f, lo, hi = inst
        assert np.all(x >= lo - 1e-7) and np.all(x <= hi + 1e-7)
        Cx = C @ x
        assert np.all(Cx >= d - 1e-7) and np.all(Cx <= f + 1e-7)
        np.testing.assert_allclose(A @ x, b, atol=1e-7)
        solved += 1
    assert solved >= 6


def test_assembled_arrowhead_full_statement_matches_highs():
    """The arrowhead LP in the full statement (block, local-link and global
    inequality rows, every bound kind), assembled monolithically by the
    oracle, has the optimal objective HiGHS finds for the same matrices."""
    from instances import general_block_lp
    for seed in (0, 3):
        inst = general.assemble_general(general_block_lp(seed))
        h = _highs(*inst)
        assert h.status == 0
        r = general.solve_general(*inst)
        assert r["status"] == "optimal"
        assert abs(r["objective"] - h.fun) <= 1e-7 * (1 + abs(h.fun)), (seed, r["objective"], h.fun)
