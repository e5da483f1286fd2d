"""Tensor-core (tcgen05) trailing updates of the FP32 block factors.

The update C_IJ -= L_Ik L_Jk' of the batched partial Cholesky runs on the
tensor cores with TF32 hi/lo split operands (hi*hi + hi*lo + lo*hi, FP32
accumulation).  Checked on shapes whose blocks span several 64-row tiles
with ragged last tiles, odd and even trailing tile counts and partial last
pivot tiles:
  * block by block, the partially factored augmented matrix agrees with the
    FP32-pipe kernel's to FP32-level accuracy (relative to the block's
    scale), and both agree with the oracle's Schur complement;
  * directions solved with these factors as the preconditioner reach the
    1e-10 Newton residual of the unregularised system and match the
    oracle's dense direction;
  * a mixed-precision IPM using them reaches the oracle's optimum.
"""
import numpy as np
import pytest

from instances import random_block_lp
from oracle import ipm as oipm
from oracle import lp as olp
from oracle import newton as onewton
from oracle import schur as oschur

pytestmark = pytest.mark.gpu

SHAPES = {
    "ragged_multi": dict(N=4, m_sizes=[300, 517, 64, 130], n_sizes=[450, 700, 96, 200],
                         nnz_per_col=5, n0=6, w_density=0.1, l=[5, 3, 7], mg=2, global_nnz=6,
                         x0_link_nnz=2, x0_global_nnz=2),
    "even_odd_tiles": dict(N=3, m_sizes=[383, 384, 449], n_sizes=[570, 576, 680],
                           nnz_per_col=6, n0=1, w_density=0.3, l=[20, 20], mg=0),
}


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_07731_gb300 as P
    return P


def _point(lp, seed, spread=1.0):
    A, b, c = olp.assemble(lp)
    rng = np.random.default_rng(seed)
    n, m = A.shape[1], A.shape[0]
    x = np.exp(spread * rng.standard_normal(n))
    z = np.exp(spread * rng.standard_normal(n))
    return A, x, z, rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n)


def _fp32(P, update, **kw):
    return P.default_options(precision=P.PREC_MIXED, fp32_cond_max=1e300, fp32_update=update,
                             **kw)


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_tensor_core_factor_matches_fp32_pipe(P, name):
    from paper_2412_07731_gb300._lib import kkt_block_factor_dense
    lp = random_block_lp(7, **SHAPES[name])
    A, x, z, *_ = _point(lp, 3, 0.5)
    ptc = P.arrowhead_lp_create(lp, _fp32(P, 2))
    pcc = P.arrowhead_lp_create(lp, _fp32(P, 1))
    P.kkt_factor(ptc, x, z, 0.0, 0.0)
    P.kkt_factor(pcc, x, z, 0.0, 0.0)
    for i in range(lp.N):
        Ft = kkt_block_factor_dense(ptc, i)
        Fc = kkt_block_factor_dense(pcc, i)
        scale = np.abs(Fc).max()
        assert np.abs(Ft - Fc).max() <= 2e-5 * scale, (i, np.abs(Ft - Fc).max() / scale)
    S_ref = oschur.schur_reduced(lp, x, z)
    for prob in (ptc, pcc):
        S = P.kkt_schur_dense(prob)
        assert np.abs(S - S_ref).max() <= 1e-4 * np.abs(S_ref).max()
    ptc.close()
    pcc.close()


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_tensor_core_direction_matches_oracle(P, name):
    lp = random_block_lp(8, **SHAPES[name])
    A, x, z, rd, rp, rc = _point(lp, 4)
    prob = P.arrowhead_lp_create(lp, _fp32(P, 2))
    P.kkt_factor(prob, x, z)
    (dx, dy, dz), info = P.kkt_solve(prob, rd, rp, rc)
    res = onewton.relative_residual(A, x, z, dx, dy, dz, rd, rp, rc)
    assert res < 1e-10, (res, info)
    ex, ey, ez = onewton.direction_dense(A, x, z, rd, rp, rc)
    got = np.concatenate([dx, dy, dz])
    ref = np.concatenate([ex, ey, ez])
    J = onewton.newton_matrix_dense(A, x, z)
    bound = max(1e-9, 1e-13 * np.linalg.cond(J))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < bound
    prob.close()


def test_tensor_core_ipm_reaches_oracle_optimum(P):
    lp = random_block_lp(9, **SHAPES["ragged_multi"])
    A, b, c = olp.assemble(lp)
    ref = oipm.solve(A, b, c)
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=P.PREC_MIXED, fp32_update=2))
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0 and r["factors_fp32"] > 0
    assert abs(r["pobj"] - ref["pobj"]) / (1 + abs(ref["pobj"])) <= 1e-8
    prob.close()


def test_persistent_update_matches_per_tile_update(P):
    """The persistent pipelined kernel (one CTA per SM walking the step's
    output tiles, two operand stages and two TMEM accumulators in flight)
    issues the same products in the same order as the one-CTA-per-tile
    kernel, and each output tile is reduced into C by exactly one job per
    step, so the two factors agree bit for bit.  40 blocks of about nine
    tiles give several hundred jobs per step: each CTA runs several, so both
    stages and both accumulators are reused across mbarrier phases."""
    from paper_2412_07731_gb300._lib import kkt_block_factor_dense
    N = 40
    rng = np.random.default_rng(5)
    m = [int(v) for v in rng.integers(420, 560, N)]
    n = [int(1.4 * v) for v in m]
    lp = random_block_lp(11, N=N, m_sizes=m, n_sizes=n, nnz_per_col=5, n0=4, w_density=0.2,
                         l=[4] * (N - 1), mg=2, global_nnz=4)
    A, x, z, *_ = _point(lp, 6, 0.5)
    probs = {u: P.arrowhead_lp_create(lp, _fp32(P, u)) for u in (2, 3)}
    probs[0] = P.arrowhead_lp_create(lp)   # FP64 factors
    for prob in probs.values():
        P.kkt_factor(prob, x, z, 0.0, 0.0)
    for i in range(N):
        F2 = kkt_block_factor_dense(probs[2], i)
        F3 = kkt_block_factor_dense(probs[3], i)
        assert np.array_equal(F2, F3), i
        # FP32-level accuracy against the FP64 factor, relative to the block's
        # scale (hi + lo carries 22 of x's 24 bits and lo*lo is dropped, so
        # the split product's error exceeds the FP32 pipe's by up to ~20x;
        # the Schur corner carries the cancellation of C - G' M^-1 G, and the
        # worst block here sits at 3e-5)
        F64 = kkt_block_factor_dense(probs[0], i)
        e3 = np.abs(F3 - F64).max()
        assert e3 <= 1e-4 * np.abs(F64).max(), (i, e3)
    S_ref = oschur.schur_reduced(lp, x, z)
    S = P.kkt_schur_dense(probs[3])
    assert np.abs(S - S_ref).max() <= 1e-4 * np.abs(S_ref).max()
    for prob in probs.values():
        prob.close()


def test_persistent_update_ipm_reaches_oracle_optimum(P):
    lp = random_block_lp(9, **SHAPES["ragged_multi"])
    A, b, c = olp.assemble(lp)
    ref = oipm.solve(A, b, c)
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=P.PREC_MIXED, fp32_update=3))
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0 and r["factors_fp32"] > 0
    assert abs(r["pobj"] - ref["pobj"]) / (1 + abs(ref["pobj"])) <= 1e-8
    prob.close()


# ---------------------------------------------------------------------------
# float-float factors: exact FP16 digit products on the tensor cores
# ---------------------------------------------------------------------------
def _ff(P, update, **kw):
    return P.default_options(precision=P.PREC_MIXED, fp32_cond_max=1.0, ff_update=update, **kw)


def test_persistent_digit_update_matches_per_tile_update(P):
    """The persistent digit-product kernel (two K-half operand stages, the
    C tile reloaded after each store) sums the same exact integer products
    D_q, only in another order, so its float-float factor equals the
    one-CTA-per-tile kernel's bit for bit; several hundred jobs per step
    give each CTA several jobs.  Both stay near the FP64 factor."""
    from paper_2412_07731_gb300._lib import kkt_block_factor_dense
    N = 40
    rng = np.random.default_rng(6)
    m = [int(v) for v in rng.integers(420, 560, N)]
    n = [int(1.4 * v) for v in m]
    lp = random_block_lp(12, N=N, m_sizes=m, n_sizes=n, nnz_per_col=5, n0=4, w_density=0.2,
                         l=[4] * (N - 1), mg=2, global_nnz=4)
    A, x, z, *_ = _point(lp, 7, 2.0)
    probs = {u: P.arrowhead_lp_create(lp, _ff(P, u)) for u in (2, 3)}
    p64 = P.arrowhead_lp_create(lp)
    for prob in list(probs.values()) + [p64]:
        P.kkt_factor(prob, x, z, 0.0, 0.0)
    for i in range(N):
        F2 = kkt_block_factor_dense(probs[2], i)
        F3 = kkt_block_factor_dense(probs[3], i)
        assert np.array_equal(F2, F3), i
        F64 = kkt_block_factor_dense(p64, i)
        assert np.abs(F3 - F64).max() <= 1e-8 * np.abs(F64).max(), i
    for prob in list(probs.values()) + [p64]:
        prob.close()


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_digit_float_float_factor_matches_double_float(P, name):
    """At a point where D spans ~1e10, block by block, the float-float factor
    of the digit-product update is nearly as close to the FP64 factor as the
    double-float FP32-pipe update's is (within 10x, and below 1e-8 of the
    block's scale: the per-row digit scaling keeps 49 bits relative to the
    row's largest entry, not to each entry), and both give the oracle's Schur
    complement to 1e-8 of its scale at this point (FP64 factors: ~1e-10;
    FP32 factors reach only ~1e-5)."""
    from paper_2412_07731_gb300._lib import kkt_block_factor_dense
    lp = random_block_lp(10, **SHAPES[name])
    A, x, z, *_ = _point(lp, 5, 3.0)
    poz = P.arrowhead_lp_create(lp, _ff(P, 2))
    pdf = P.arrowhead_lp_create(lp, _ff(P, 1))
    p64 = P.arrowhead_lp_create(lp)
    for prob in (poz, pdf, p64):
        P.kkt_factor(prob, x, z, 0.0, 0.0)
    for i in range(lp.N):
        F64 = kkt_block_factor_dense(p64, i)
        scale = np.abs(F64).max()
        e_oz = np.abs(kkt_block_factor_dense(poz, i) - F64).max() / scale
        e_dd = np.abs(kkt_block_factor_dense(pdf, i) - F64).max() / scale
        assert e_oz <= max(10.0 * e_dd, 1e-12) and e_oz <= 1e-8, (i, e_oz, e_dd)
    S_ref = oschur.schur_reduced(lp, x, z)
    for prob in (poz, pdf):
        S = P.kkt_schur_dense(prob)
        assert np.abs(S - S_ref).max() <= 1e-8 * np.abs(S_ref).max()
    for prob in (poz, pdf, p64):
        prob.close()


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_digit_float_float_direction_matches_oracle(P, name):
    lp = random_block_lp(11, **SHAPES[name])
    A, x, z, rd, rp, rc = _point(lp, 6, 2.0)
    prob = P.arrowhead_lp_create(lp, _ff(P, 2))
    P.kkt_factor(prob, x, z)
    (dx, dy, dz), info = P.kkt_solve(prob, rd, rp, rc)
    res = onewton.relative_residual(A, x, z, dx, dy, dz, rd, rp, rc)
    assert res < 1e-10, (res, info)
    assert info["refine_steps"] <= 3, info   # the factor is nearly exact
    ex, ey, ez = onewton.direction_dense(A, x, z, rd, rp, rc)
    got = np.concatenate([dx, dy, dz])
    ref = np.concatenate([ex, ey, ez])
    J = onewton.newton_matrix_dense(A, x, z)
    bound = max(1e-9, 1e-13 * np.linalg.cond(J))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < bound
    prob.close()


def test_digit_float_float_ipm_reaches_oracle_optimum(P):
    lp = random_block_lp(12, **SHAPES["ragged_multi"])
    A, b, c = olp.assemble(lp)
    ref = oipm.solve(A, b, c)
    prob = P.arrowhead_lp_create(lp, _ff(P, 2))
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0 and r["factors_ff"] > 0
    assert abs(r["pobj"] - ref["pobj"]) / (1 + abs(ref["pobj"])) <= 1e-8
    prob.close()


def test_autotune_picks_a_kernel_and_solves(P):
    """The autotuner times each trailing-update kernel on the handle's own
    blocks, keeps the faster per precision, and the handle then solves to the
    oracle's optimum with its choice."""
    lp = random_block_lp(13, **SHAPES["ragged_multi"])
    A, b, c = olp.assemble(lp)
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=P.PREC_MIXED))
    t = P.autotune(prob)
    assert all(t[k] > 0 for k in ("fp32_tensor_ms", "fp32_pipe_ms", "ff_tensor_ms", "ff_pipe_ms",
                                  "fp32_tensor_persistent_ms", "ff_tensor_persistent_ms"))
    assert t["fp32_update"] in (1, 2, 3) and t["ff_update"] in (1, 2, 3)
    (x, y, z), r = P.ipm_solve(prob)
    ref = oipm.solve(A, b, c)
    assert r["status"] == 0
    assert abs(r["pobj"] - ref["pobj"]) / (1 + abs(ref["pobj"])) <= 1e-8
    prob.close()
