"""Pins of the Schur-complement decomposition (Alg. 1-3, App. A)."""
import numpy as np
import pytest

from instances import random_block_lp, config0
from oracle import schur, newton, lp as lpm


def _lp(seed, mg=2, x0_link=1):
    return random_block_lp(seed, N=5, m_sizes=[6, 5, 7, 6, 4], n_sizes=[10, 9, 11, 10, 8],
                           nnz_per_col=2, n0=3, w_density=0.5, l=[2, 1, 3, 2],
                           link_nnz=(2, 2), mg=mg, global_nnz=3, x0_link_nnz=x0_link,
                           x0_global_nnz=1)


def _pt(lp, seed=0):
    A, b, c = lpm.assemble(lp)
    rng = np.random.default_rng(seed)
    n, m = A.shape[1], A.shape[0]
    return (A, np.exp(rng.standard_normal(n)), np.exp(rng.standard_normal(n)),
            rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_alg3_equals_monolithic(seed):
    lp = _lp(seed)
    A, x, z, rd, rp, rc = _pt(lp, seed)
    d_mono = newton.direction_dense(A, x, z, rd, rp, rc)
    d_alg3 = schur.solve_alg3(lp, x, z, rd, rp, rc)
    for u, v in zip(d_mono, d_alg3):
        np.testing.assert_allclose(u, v, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("seed", [0, 3])
def test_app_a_formulas_equal_alg1(seed):
    lp = _lp(seed)
    A, x, z, *_ = _pt(lp, seed)
    S = schur.schur_alg1(lp, x, z)
    _, _, K0 = schur.paper_blocks(lp, x, z)
    contrib = K0 - S
    p = schur.app_a_perm(lp)
    np.testing.assert_allclose(schur.app_a_contrib(lp, x, z), contrib[np.ix_(p, p)],
                               rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("seed", [0, 4])
def test_reduced_normal_form_equals_alg1(seed):
    """Normal-equation Schur complement == Alg. 1's on the augmented blocks."""
    lp = _lp(seed)
    A, x, z, *_ = _pt(lp, seed)
    S = schur.schur_alg1(lp, x, z)
    q = schur.reduced_perm(lp)
    np.testing.assert_allclose(schur.schur_reduced(lp, x, z), S[np.ix_(q, q)],
                               rtol=1e-9, atol=1e-10)


def test_zero_pattern_and_observation1():
    """Outside block-tridiagonal + border, the contributions are exact zeros."""
    lp = _lp(5, x0_link=0)
    A, x, z, *_ = _pt(lp, 5)
    S = schur.schur_alg1(lp, x, z)
    _, _, K0 = schur.paper_blocks(lp, x, z)
    contrib = (K0 - S)[np.ix_(schur.app_a_perm(lp), schur.app_a_perm(lp))]
    lo = lp.link_offsets()
    nl = int(lo[-1])
    allowed = np.zeros_like(contrib, dtype=bool)
    allowed[nl:, :] = True
    allowed[:, nl:] = True
    for j in range(lp.N - 1):
        for k in (j - 1, j, j + 1):
            if 0 <= k < lp.N - 1:
                allowed[lo[j]:lo[j + 1], lo[k]:lo[k + 1]] = True
    assert np.all(contrib[~allowed] == 0.0)
    nnz = int(np.count_nonzero(S))
    assert nnz <= schur.observation1_bound(lp)
    # in general position every allowed block is dense: the bound is attained
    assert np.count_nonzero(contrib) == schur.observation1_bound(lp)


def test_schur_symmetric_quasidefinite():
    """x_0 part negative definite, link part positive definite (Sec. 2.3 signs)."""
    lp = _lp(6, mg=0)
    A, x, z, *_ = _pt(lp, 6)
    Sr = schur.schur_reduced(lp, x, z)
    np.testing.assert_allclose(Sr, Sr.T, atol=1e-10)
    nl = int(lp.link_offsets()[-1])
    assert np.all(np.linalg.eigvalsh(Sr[:nl, :nl]) > 0)
    assert np.all(np.linalg.eigvalsh(Sr[nl:, nl:]) < 0)
