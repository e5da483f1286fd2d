"""The seeded synthetic workloads: shapes as stated, planted optima valid.

  * the uneven workload's blocks: m_i in {500..4000}, n_i = floor(1.5 m_i),
    8 nonzeros per column of A_i, 100 linking variables, 16 link rows per
    pair;
  * the block-by-block nondegenerate plant (the batch workload's): |B| = m,
    x* >= 0 and z* >= 0 strictly complementary, A x* = b, A'y* + z* = c, A_B
    nonsingular (sparse LU with a bounded 1-norm condition estimate), and the
    oracle's IPM finds x* on small instances (the optimum is unique).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from instances import config2, random_block_lp
from oracle import ipm as oipm
from oracle import lp as olp


def test_uneven_workload_shapes():
    lp = config2(2, N=16)
    assert lp.N == 16 and lp.n0 == 100 and np.all(np.asarray(lp.l) == 16)
    for A in lp.A:
        m, n = A.shape
        assert 500 <= m <= 4000 and n == (3 * m) // 2
        assert np.all(np.diff(sp.csc_matrix(A).indptr) == 8)


def _check_plant(lp):
    A, b, c = olp.assemble(lp)
    x, y, z = lp.xstar, lp.ystar, lp.zstar
    m, n = A.shape
    B = lp.basis
    assert len(B) == m and len(np.unique(B)) == m
    assert np.all(x >= 0) and np.all(z >= 0)
    assert np.all(x[B] >= 0.1) and np.count_nonzero(x) == m
    assert np.max(np.abs(x * z)) == 0.0
    assert np.all(np.delete(z, B) >= 0.1)
    assert np.linalg.norm(A @ x - b) <= 1e-10 * (1 + np.linalg.norm(b))
    assert np.linalg.norm(A.T @ y + z - c) <= 1e-10 * (1 + np.linalg.norm(c))
    AB = sp.csc_matrix(A[:, B])
    lu = spla.splu(AB)
    op = spla.LinearOperator(AB.shape, matvec=lu.solve, rmatvec=lambda v: lu.solve(v, "T"),
                             dtype=float)
    cond1 = spla.norm(AB, 1) * spla.onenormest(op)
    assert np.isfinite(cond1) and cond1 < 1e12, cond1
    return A, b, c


@pytest.mark.parametrize("seed", [4, 5])
def test_block_basis_plant_of_the_batch_workload(seed):
    _check_plant(config2(seed, N=8, nondegenerate=True))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_block_basis_plant_is_the_unique_optimum(seed):
    lp = random_block_lp(seed, N=4, m_sizes=[30, 45, 25, 40], n_sizes=[45, 70, 40, 60],
                         nnz_per_col=5, n0=3, w_density=0.2, l=[3, 2, 4], mg=1, global_nnz=4,
                         plant="basis_blocks")
    A, b, c = _check_plant(lp)
    r = oipm.solve(A, b, c)
    assert r["status"] == "optimal"
    # an IPM iterate at relative gap 1e-8 sits within ~1e-6 of the vertex
    assert np.abs(r["x"] - lp.xstar).max() <= 1e-5 * max(1.0, np.abs(lp.xstar).max())
    assert abs(r["pobj"] - float(c @ lp.xstar)) <= 1e-8 * (1 + abs(float(c @ lp.xstar)))
