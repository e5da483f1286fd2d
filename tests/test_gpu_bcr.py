"""Block cyclic reduction of the link chain (the block-tridiagonal part of
the Schur complement, App. A) against the sequential chain Cholesky and the
oracle.

Both chain factorisations solve the same Schur system, so the directions
they give must agree with each other and with the oracle's monolithic
Newton system (relative residual 1e-10).  Shapes: a 300-pair chain (nine
levels, a ragged last level), link blocks above 32 rows (the general
Cholesky path), link blocks of different sizes along the chain, and a batch
whose LPs make separate chain segments.
"""
import numpy as np
import pytest

from instances import random_block_lp
from oracle import newton as onewton
from oracle import lp as olp
from oracle import schur as oschur

pytestmark = pytest.mark.gpu

SHAPES = {
    "chain_300": dict(N=301, m_sizes=[12] * 301, n_sizes=[18] * 301, nnz_per_col=3, n0=3,
                      w_density=0.3, l=5, link_nnz=(3, 3), mg=1, global_nnz=4,
                      x0_link_nnz=1, x0_global_nnz=1),
    "wide_links": dict(N=6, m_sizes=[90, 80, 100, 85, 95, 70], n_sizes=[140, 130, 150, 130, 140, 110],
                       nnz_per_col=5, n0=4, w_density=0.2, l=[40, 33, 48, 36, 41], mg=1,
                       global_nnz=6, x0_link_nnz=2, x0_global_nnz=2),
    "uneven_links": dict(N=12, m_sizes=[40] * 12, n_sizes=[60] * 12, nnz_per_col=4, n0=2,
                         w_density=0.3, l=[1, 7, 3, 12, 5, 2, 9, 4, 6, 1, 8], mg=0),
}


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_07731_gb300 as P
    return P


def _point(lp, seed):
    A, b, c = olp.assemble(lp)
    rng = np.random.default_rng(seed)
    n, m = A.shape[1], A.shape[0]
    return (A, np.exp(rng.standard_normal(n)), np.exp(rng.standard_normal(n)),
            rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n))


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_cyclic_reduction_direction(P, name):
    lp = random_block_lp(31, **SHAPES[name])
    A, x, z, rd, rp, rc = _point(lp, 2)
    dirs = {}
    for chain in (0, 1):
        prob = P.arrowhead_lp_create(lp, P.default_options(schur_chain=chain))
        P.kkt_factor(prob, x, z)
        (dx, dy, dz), info = P.kkt_solve(prob, rd, rp, rc)
        res = onewton.relative_residual(A, x, z, dx, dy, dz, rd, rp, rc)
        assert res < 1e-10, (chain, res, info)
        dirs[chain] = np.concatenate([dx, dy, dz])
        prob.close()
    assert np.linalg.norm(dirs[0] - dirs[1]) <= 1e-9 * np.linalg.norm(dirs[1])


def test_cyclic_reduction_preconditioner_alone(P):
    """Without Krylov refinement the solve is the factor's own solve: with
    delta = 0 both chain factorisations give the exact Schur solve, so the
    unrefined directions agree with the oracle's to rounding."""
    lp = random_block_lp(32, **SHAPES["uneven_links"])
    A, x, z, rd, rp, rc = _point(lp, 3)
    ex, ey, ez = onewton.direction_dense(A, x, z, rd, rp, rc)
    ref = np.concatenate([ex, ey, ez])
    for chain in (0, 1):
        prob = P.arrowhead_lp_create(lp, P.default_options(schur_chain=chain, refine_max=0))
        P.kkt_factor(prob, x, z, 0.0, 0.0)
        (dx, dy, dz), _ = P.kkt_solve(prob, rd, rp, rc)
        got = np.concatenate([dx, dy, dz])
        assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref), chain
        S = P.kkt_schur_dense(prob)
        S_ref = oschur.schur_reduced(lp, x, z)
        assert np.abs(S - S_ref).max() <= 1e-11 * np.abs(S_ref).max()
        prob.close()


def test_cyclic_reduction_batch_segments(P):
    lps = [random_block_lp(40 + k, N=9, m_sizes=[30] * 9, n_sizes=[45] * 9, nnz_per_col=4,
                           n0=2, w_density=0.3, l=[3, 4, 2, 5, 3, 4, 2, 3], mg=1,
                           global_nnz=3, x0_link_nnz=1, x0_global_nnz=1) for k in range(3)]
    prob = P.arrowhead_lp_create(lps, P.default_options(schur_chain=0))
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0
    for (ix, _), q in zip(P.batch_layout(lps), lps):
        A, b, c = olp.assemble(q)
        obj = float(c @ q.xstar)
        assert abs(float(c @ x[ix]) - obj) <= 1e-8 * (1 + abs(obj))
    prob.close()
