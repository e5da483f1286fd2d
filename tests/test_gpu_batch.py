"""Batched independent LPs (batch > 1): one handle solves their direct sum.

Pins: every LP of a batch reaches its own oracle optimum (objective within
1e-8, its own infeasibilities small); a batched KKT direction is, LP by LP,
the oracle's monolithic direction; objective gradients through LPSolve are
each LP's planted solution.
"""
import numpy as np
import pytest

from instances import config0, config2, random_block_lp, tiny_lp
from oracle import ipm as oipm
from oracle import lp as olp
from oracle import newton as onewton

pytestmark = pytest.mark.gpu

SHAPE = dict(N=5, m_sizes=[1, 63, 64, 65, 130], n_sizes=[3, 95, 96, 100, 200], nnz_per_col=3,
             n0=4, w_density=0.2, l=[2, 3, 1, 4], mg=2, global_nnz=4, x0_link_nnz=2,
             x0_global_nnz=2)


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_07731_gb300 as P
    return P


def _mixed_batch():
    return [config0(0), random_block_lp(3, **SHAPE), tiny_lp(5, N=3, m=2, n=4, n0=1, l=1, mg=1),
            config0(4)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_reaches_every_oracle_optimum(P, prec):
    lps = _mixed_batch()
    opts = P.default_options(precision=P.PREC_MIXED if prec == "mixed" else P.PREC_FP64)
    prob = P.arrowhead_lp_create(lps, opts)
    (x, y, z), r = P.ipm_solve(prob)
    assert r["rel_gap"] <= 1e-8 and r["pinf"] <= 1e-8 and r["dinf"] <= 1e-8
    for q, (ix, iy) in zip(lps, P.batch_layout(lps)):
        A, b, c = olp.assemble(q)
        ref = oipm.solve(A, b, c)
        xb, yb, zb = x[ix], y[iy], z[ix]
        assert abs(c @ xb - ref["pobj"]) <= 1e-8 * (1 + abs(ref["pobj"]))
        assert np.abs(A @ xb - b).max() <= 1e-7 * (1 + np.abs(b).max())
        assert np.abs(A.T @ yb + zb - c).max() <= 1e-7 * (1 + np.abs(c).max())
    prob.close()


def test_batch_direction_matches_oracle_per_lp(P):
    lps = _mixed_batch()
    lay = P.batch_layout(lps)
    prob = P.arrowhead_lp_create(lps)
    rng = np.random.default_rng(7)
    n, m = prob.n, prob.m
    x, z = np.exp(rng.standard_normal(n)), np.exp(rng.standard_normal(n))
    rd, rp, rc = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n)
    P.kkt_factor(prob, x, z)
    (dx, dy, dz), info = P.kkt_solve(prob, rd, rp, rc)
    for q, (ix, iy) in zip(lps, lay):
        A, _, _ = olp.assemble(q)
        res = onewton.relative_residual(A, x[ix], z[ix], dx[ix], dy[iy], dz[ix], rd[ix], rp[iy],
                                        rc[ix])
        assert res < 1e-10, (res, info)
    prob.close()


def test_batch_objective_gradients(P):
    torch = pytest.importorskip("torch")
    from paper_2412_07731_gb300.autograd import lp_solve
    lps = [random_block_lp(s, N=4, m_sizes=[40] * 4, n_sizes=[60] * 4, nnz_per_col=6, n0=3,
                           w_density=1.0, l=2, link_nnz=(5, 5), mg=0, plant="nondegenerate")
           for s in (21, 22, 23)]
    lay = P.batch_layout(lps)
    prob = P.arrowhead_lp_create(lps)
    c = np.zeros(prob.n)
    b = np.zeros(prob.m)
    for q, (ix, iy) in zip(lps, lay):
        c[ix] = q.c_global()
        b[iy] = q.b_global()
    dev = torch.device("cuda", 0)
    ct = torch.tensor(c, dtype=torch.float64, device=dev, requires_grad=True)
    bt = torch.tensor(b, dtype=torch.float64, device=dev, requires_grad=True)
    x, _, _ = lp_solve(ct, bt, prob)
    (ct * x).sum().backward()
    gc, gb = ct.grad.cpu().numpy(), bt.grad.cpu().numpy()
    for q, (ix, iy) in zip(lps, lay):
        assert np.abs(gc[ix] - q.xstar).max() <= 1e-6
        assert np.abs(gb[iy] - q.ystar).max() <= 1e-6
    prob.close()


def test_batch_of_uneven_block_lps(P):
    """Four LPs of the uneven-block shape (blocks of 500..4000 rows, 100
    linking variables, 16 links per pair) with 8 blocks each, in mixed
    precision: each reaches its planted objective."""
    lps = [config2(seed, N=8) for seed in (4, 5, 6, 7)]
    prob = P.arrowhead_lp_create(lps, P.default_options(precision=P.PREC_MIXED))
    (x, y, z), r = P.ipm_solve(prob)
    for q, (ix, _) in zip(lps, P.batch_layout(lps)):
        obj = float(q.c_global() @ q.xstar)
        assert abs(float(q.c_global() @ x[ix]) - obj) <= 1e-8 * (1 + abs(obj))
    prob.close()
