"""pivot_mode = 1: failing pivots of the block factors are dropped (replaced
by a huge value, which leaves the row out of the factor) instead of clamped.

  * a block with a repeated row makes M_i = A_i D_i A_i' singular at every
    iterate: the repeated row's pivot fails in every factor, in every
    precision.  The IPM still reaches the optimum that scipy's HiGHS finds
    for the assembled LP (the Krylov refinement solves the exact Newton
    system; the repeated row's dual is not unique, the objective is);
  * on a full-rank LP the mixed-precision IPM in drop mode reaches the
    oracle's optimum, like the clamping mode.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from instances import random_block_lp
from oracle import ipm as oipm
from oracle import lp as olp

pytestmark = pytest.mark.gpu

SHAPE = dict(N=4, m_sizes=[300, 517, 64, 130], n_sizes=[450, 700, 96, 200], nnz_per_col=5,
             n0=6, w_density=0.1, l=[5, 3, 7], mg=2, global_nnz=6, x0_link_nnz=2,
             x0_global_nnz=2)


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_07731_gb300 as P
    return P


def _rel(a, b):
    return abs(a - b) / (1.0 + abs(b))


def _repeat_row(lp, blk, row):
    """The LP with row `row` of block `blk` (A_i, W_i and b_i) appended again."""
    A = sp.csr_matrix(lp.A[blk])
    W = sp.csr_matrix(lp.W[blk])
    lp.A[blk] = sp.vstack([A, A[row]]).tocsc()
    lp.W[blk] = sp.vstack([W, W[row]]).tocsc()
    lp.b[blk] = np.concatenate([lp.b[blk], lp.b[blk][row:row + 1]])
    lp.xstar = lp.ystar = lp.zstar = None
    return lp


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_repeated_row_reaches_highs_optimum(P, prec):
    from scipy.optimize import linprog
    lp = _repeat_row(random_block_lp(21, **SHAPE), 1, 7)
    A, b, c = olp.assemble(lp)
    ref = linprog(c, A_eq=A, b_eq=b, bounds=(0, None), method="highs")
    assert ref.status == 0
    precision = P.PREC_FP64 if prec == "fp64" else P.PREC_MIXED
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=precision, pivot_mode=1))
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0, r
    assert r["tiny_pivots"] > 0   # the repeated row's pivot failed
    assert _rel(r["pobj"], ref.fun) <= 1e-7
    m = olp.measures(A, b, c, x, y, z)
    assert m["pinf"] <= 1e-8 and m["gap"] <= 1e-8
    prob.close()


def test_drop_mode_mixed_reaches_oracle_optimum(P):
    lp = random_block_lp(22, **SHAPE)
    A, b, c = olp.assemble(lp)
    ref = oipm.solve(A, b, c)
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=P.PREC_MIXED, pivot_mode=1))
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0
    assert _rel(r["pobj"], ref["pobj"]) <= 1e-8
    prob.close()
