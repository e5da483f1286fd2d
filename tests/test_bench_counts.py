"""The algorithmic work bench.py divides by in its rooflines.

block_factor_flops: the flop count of one batched partial Cholesky of the
augmented block matrices, pinned against an explicit count of the divisions
and multiply-adds of a column-by-column partial Cholesky on small blocks
(and checked to give that factorisation, against scipy's Cholesky)."""
import numpy as np
import pytest

import bench
from instances import random_block_lp


def _partial_cholesky_count(M, p):
    """Right-looking partial Cholesky of M over its first p pivots, counting a
    division as 1 flop and a multiply-add as 2 (the square roots not counted)."""
    a = M.shape[0]
    L = np.tril(M.astype(float))
    flops = 0
    for c in range(p):
        L[c, c] = np.sqrt(L[c, c])
        for r in range(c + 1, a):
            L[r, c] /= L[c, c]
            flops += 1
        for r in range(c + 1, a):
            for s in range(c + 1, r + 1):
                L[r, s] -= L[r, c] * L[s, c]
                flops += 2
    return L, flops


@pytest.mark.parametrize("seed", [0, 1])
def test_block_factor_flops_is_the_partial_cholesky_count(seed):
    lp = random_block_lp(seed, N=3, m_sizes=[5, 7, 4], n_sizes=[8, 10, 6], nnz_per_col=2, n0=2,
                         w_density=0.5, l=[2, 3], mg=1, global_nnz=2)
    rng = np.random.default_rng(seed)
    total = 0
    for i, A in enumerate(lp.A):
        m = A.shape[0]
        k = lp.n0 + lp.mg + (int(lp.l[i - 1]) if i > 0 else 0) + (int(lp.l[i]) if i < lp.N - 1 else 0)
        a = m + k
        B = rng.standard_normal((a, a + 3))
        M = B @ B.T + a * np.eye(a)
        L, f = _partial_cholesky_count(M, m)
        np.testing.assert_allclose(np.tril(L[:m, :m]), np.linalg.cholesky(M[:m, :m]), rtol=1e-12)
        total += f
    assert bench.block_factor_flops(lp) == total
