"""Mixed precision: FP32 block factors precondition an FP64 Krylov solve of the
unregularised Newton system; the IPM switches to FP64 factors when the
preconditioner stops being good enough (the ill-conditioned end game)."""
import numpy as np
import pytest

from instances import config0, random_block_lp
from oracle import ipm as oipm
from oracle import lp as olp
from oracle import newton as onewton

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_07731_gb300 as P
    return P


def _mixed(P, **kw):
    return P.default_options(precision=P.PREC_MIXED, **kw)


SHAPE = dict(N=5, m_sizes=[1, 63, 64, 65, 130], n_sizes=[3, 95, 96, 100, 200], nnz_per_col=3,
             n0=4, w_density=0.2, l=[2, 3, 1, 4], mg=2, global_nnz=4, x0_link_nnz=2,
             x0_global_nnz=2)


@pytest.mark.parametrize("which", ["c0", "ragged"])
def test_mixed_direction_reaches_fp64_residual(P, which):
    lp = config0(2) if which == "c0" else random_block_lp(3, **SHAPE)
    A, b, c = olp.assemble(lp)
    rng = np.random.default_rng(1)
    n, m = A.shape[1], A.shape[0]
    x, z = np.exp(rng.standard_normal(n)), np.exp(rng.standard_normal(n))
    rd, rp, rc = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n)
    prob = P.arrowhead_lp_create(lp, _mixed(P))
    P.kkt_factor(prob, x, z)
    (dx, dy, dz), info = P.kkt_solve(prob, rd, rp, rc)
    res = onewton.relative_residual(A, x, z, dx, dy, dz, rd, rp, rc)
    assert res < 1e-10, (res, info)
    ex, ey, ez = onewton.direction_dense(A, x, z, rd, rp, rc)
    J = onewton.newton_matrix_dense(A, x, z)
    bound = max(1e-9, 1e-13 * np.linalg.cond(J))
    got = np.concatenate([dx, dy, dz])
    ref = np.concatenate([ex, ey, ez])
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < bound


def test_mixed_schur_close_to_fp64(P):
    """The Schur complement assembled from FP32 block factors agrees with the
    FP64 one to FP32 accuracy (relative to the matrix scale)."""
    lp = random_block_lp(4, **SHAPE)
    A, b, c = olp.assemble(lp)
    rng = np.random.default_rng(2)
    n = A.shape[1]
    x, z = np.exp(0.5 * rng.standard_normal(n)), np.exp(0.5 * rng.standard_normal(n))
    p64 = P.arrowhead_lp_create(lp)
    p32 = P.arrowhead_lp_create(lp, _mixed(P))
    P.kkt_factor(p64, x, z, 0.0, 0.0)
    P.kkt_factor(p32, x, z, 0.0, 0.0)
    S64, S32 = P.kkt_schur_dense(p64), P.kkt_schur_dense(p32)
    assert np.abs(S32 - S64).max() <= 1e-4 * np.abs(S64).max()


@pytest.mark.parametrize("seed", range(6))
def test_mixed_ipm_matches_fp64_objective(P, seed):
    lp = config0(seed)
    A, b, c = olp.assemble(lp)
    prob = P.arrowhead_lp_create(lp, _mixed(P))
    (x, y, z), r = P.ipm_solve(prob)
    obj = float(c @ lp.xstar)
    assert r["status"] == 0
    assert abs(r["pobj"] - obj) / (1 + abs(obj)) <= 1e-8
    m = olp.measures(A, b, c, x, y, z)
    assert m["pinf"] <= 1e-8 and m["dinf"] <= 1e-8 and m["gap"] <= 1e-8


def test_mixed_ipm_structured_shape(P):
    lp = random_block_lp(21, N=6, m_sizes=[90, 130, 70, 64, 100, 150],
                         n_sizes=[135, 195, 105, 96, 150, 225], nnz_per_col=6, n0=8,
                         w_density=0.1, l=[4, 5, 3, 6, 2], mg=2, global_nnz=6,
                         x0_link_nnz=2, x0_global_nnz=2)
    A, b, c = olp.assemble(lp)
    ref = oipm.solve(A, b, c)
    prob = P.arrowhead_lp_create(lp, _mixed(P))
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0
    assert abs(r["pobj"] - ref["pobj"]) / (1 + abs(ref["pobj"])) <= 1e-8


def test_float_float_schur_matches_fp64(P):
    """Float-float block factors (two FP32 words, double-float trailing
    updates) give the Schur complement to nearly FP64 accuracy: at a point
    where D spans ~1e10, within 1e-10 of the FP64 one (relative to its
    scale), where FP32 factors reach only ~1e-5."""
    lp = random_block_lp(4, **SHAPE)
    A, b, c = olp.assemble(lp)
    rng = np.random.default_rng(5)
    n = A.shape[1]
    x, z = np.exp(3 * rng.standard_normal(n)), np.exp(3 * rng.standard_normal(n))
    p64 = P.arrowhead_lp_create(lp)
    P.kkt_factor(p64, x, z)
    S64 = P.kkt_schur_dense(p64)
    pff = P.arrowhead_lp_create(lp, _mixed(P, fp32_cond_max=1.0))
    P.kkt_factor(pff, x, z)
    Sff = P.kkt_schur_dense(pff)
    scale = np.abs(S64).max()
    assert np.abs(Sff - S64).max() <= 1e-10 * scale
    p32 = P.arrowhead_lp_create(lp, _mixed(P, fp32_cond_max=1e300))
    P.kkt_factor(p32, x, z)
    S32 = P.kkt_schur_dense(p32)
    assert np.abs(S32 - S64).max() > 1e3 * np.abs(Sff - S64).max()   # the test can tell them apart
    for p in (p64, pff, p32):
        p.close()


@pytest.mark.parametrize("seed", [0, 4, 8])
def test_float_float_ipm_matches_oracle(P, seed):
    """Mixed IPM with every factor past the starting point in float-float
    reaches the oracle's optimum."""
    lp = config0(seed)
    ref = oipm.solve_blocklp(lp)
    prob = P.arrowhead_lp_create(lp, _mixed(P, fp32_cond_max=1.0))
    _, r = P.ipm_solve(prob)
    assert r["factors_ff"] > 0
    assert abs(r["pobj"] - ref["pobj"]) <= 1e-8 * (1 + abs(ref["pobj"]))
    prob.close()
