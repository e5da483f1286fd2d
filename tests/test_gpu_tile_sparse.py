"""Tile-sparse trailing updates (option tile_sparse) on the energy-shaped
workload, whose blocks are banded by the hourly chain: the tensor-core
updates skip the tile jobs whose product a tile-level symbolic factorisation
shows to be structurally zero.  Those jobs add exact zeros, so every block's
partial factor, the Schur complement and the direction must equal the dense
enumeration's bit for bit, for the one-CTA-per-tile and the persistent
kernels, FP32 (TF32 split) and float-float (FP16 digits) factors alike."""
import numpy as np
import pytest

from instances import config3
from oracle import lp as olp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_07731_gb300 as P
    return P


@pytest.fixture(scope="module")
def energy():
    lp = config3(days=3)
    A, b, c = olp.assemble(lp)
    rng = np.random.default_rng(3)
    n, m = A.shape[1], A.shape[0]
    pt = (np.exp(rng.standard_normal(n)), np.exp(rng.standard_normal(n)))
    rhs = (rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n))
    return lp, pt, rhs


@pytest.mark.parametrize("prec,update", [("fp32", 2), ("fp32", 3), ("ff", 2), ("ff", 3)])
def test_tile_sparse_factor_is_bitwise_dense(P, energy, prec, update):
    from paper_2412_07731_gb300._lib import kkt_block_factor_dense
    lp, (x, z), (rd, rp, rc) = energy
    kw = (dict(fp32_cond_max=1e300, fp32_update=update) if prec == "fp32"
          else dict(fp32_cond_max=1.0, ff_update=update))
    probs = [P.arrowhead_lp_create(lp, P.default_options(precision=P.PREC_MIXED, tile_sparse=s,
                                                         **kw)) for s in (0, 1)]
    dirs = []
    for prob in probs:
        P.kkt_factor(prob, x, z)
        dirs.append(P.kkt_solve(prob, rd, rp, rc)[0])
    for i in range(lp.N):
        assert np.array_equal(kkt_block_factor_dense(probs[0], i),
                              kkt_block_factor_dense(probs[1], i)), i
    assert np.array_equal(P.kkt_schur_dense(probs[0]), P.kkt_schur_dense(probs[1]))
    for u, v in zip(dirs[0], dirs[1]):
        assert np.array_equal(u, v)
    (k0, d0), (k1, d1) = (P.kkt_update_jobs(prob) for prob in probs)
    assert k0 == d0 == d1 > 0 and 0 < k1 < d1   # the tile-sparse handle left jobs out
    for prob in probs:
        prob.close()
