"""GPU parity of the KKT factor / solve against the CPU oracle, through the C ABI.

Tolerance: the decomposed FP64 solve must match the monolithic Newton
direction to a relative error of 1e-10 and leave a relative Newton residual
below 1e-10 (both measured at moderate points where cond(J) ~ 1e4..1e6, so
FP64 rounding alone gives ~1e-12).
"""
import numpy as np
import pytest

from instances import config0, random_block_lp, tiny_lp
from oracle import adjoint as oadj
from oracle import lp as olp
from oracle import newton as onewton
from oracle import schur as oschur

pytestmark = pytest.mark.gpu

TOL_DIR = 1e-10
TOL_RES = 1e-10


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


def _rel(u, v):
    return np.linalg.norm(u - v) / max(np.linalg.norm(v), 1e-300)


SHAPES = {
    # name: kwargs of random_block_lp
    "c0": None,
    "one_block": dict(N=1, m_sizes=[70], n_sizes=[110], nnz_per_col=4, n0=5, w_density=0.3,
                      l=[], mg=2, global_nnz=5, x0_global_nnz=2),
    "ragged_tiles": dict(N=5, m_sizes=[1, 63, 64, 65, 130], n_sizes=[3, 95, 96, 100, 200],
                         nnz_per_col=3, n0=4, w_density=0.2, l=[2, 3, 1, 4], mg=2,
                         global_nnz=4, x0_link_nnz=2, x0_global_nnz=2),
    "no_border": dict(N=4, m_sizes=[50, 70, 40, 66], n_sizes=[80, 100, 60, 90], nnz_per_col=4,
                      n0=0, w_density=0.0, l=[3, 0, 5], mg=0),
    "wide_border": dict(N=3, m_sizes=[120, 129, 127], n_sizes=[180, 190, 185], nnz_per_col=5,
                        n0=70, w_density=0.1, l=[6, 7], mg=3, global_nnz=6, x0_link_nnz=3,
                        x0_global_nnz=3),
    "multi_tile": dict(N=3, m_sizes=[300, 257, 200], n_sizes=[450, 400, 310], nnz_per_col=6,
                       n0=10, w_density=0.05, l=[20, 20], mg=1, global_nnz=8),
    # link blocks above 32 rows take the general one-CTA link chain
    "long_links": dict(N=3, m_sizes=[90, 80, 100], n_sizes=[140, 130, 150], nnz_per_col=5,
                       n0=6, w_density=0.1, l=[40, 33], mg=2, global_nnz=5),
    # a small link block inside a chain that takes the general kernel
    "mixed_links": dict(N=4, m_sizes=[90, 60, 80, 100], n_sizes=[140, 95, 130, 150],
                        nnz_per_col=5, n0=6, w_density=0.1, l=[40, 8, 33], mg=2, global_nnz=5),
    # link blocks of exactly 32 rows (the register path's limit) next to a 1-row one
    "links_32": dict(N=4, m_sizes=[70, 64, 75, 66], n_sizes=[110, 100, 120, 100],
                     nnz_per_col=5, n0=5, w_density=0.1, l=[32, 1, 32], mg=1, global_nnz=4),
}


def _make(name, seed=0):
    if name == "c0":
        return config0(seed)
    return random_block_lp(seed, **SHAPES[name])


@pytest.mark.parametrize("name", list(SHAPES))
def test_schur_matches_oracle(P, name):
    lp = _make(name)
    A, x, z, *_ = _point(lp, 1)
    prob = P.arrowhead_lp_create(lp)
    P.kkt_factor(prob, x, z, 0.0, 0.0)
    S = P.kkt_schur_dense(prob)
    S_ref = oschur.schur_reduced(lp, x, z)
    assert S.shape == S_ref.shape
    scale = max(np.abs(S_ref).max(), 1.0)
    np.testing.assert_allclose(S, S_ref, rtol=0, atol=1e-11 * scale)


def _tight(P):
    # forward-error comparisons need the Krylov refinement run to the
    # rounding floor, not just to the 1e-10 residual target
    return P.default_options(refine_tol=1e-14)


@pytest.mark.parametrize("name", list(SHAPES))
def test_direction_matches_oracle(P, name):
    lp = _make(name)
    A, x, z, rd, rp, rc = _point(lp, 2)
    prob = P.arrowhead_lp_create(lp, _tight(P))
    P.kkt_factor(prob, x, z)
    (dx, dy, dz), info = P.kkt_solve(prob, rd, rp, rc)
    ex, ey, ez = onewton.direction_dense(A, x, z, rd, rp, rc)
    assert _rel(dx, ex) < TOL_DIR
    assert _rel(dy, ey) < TOL_DIR
    assert _rel(dz, ez) < TOL_DIR
    assert onewton.relative_residual(A, x, z, dx, dy, dz, rd, rp, rc) < TOL_RES
    assert info["rel_residual"] < TOL_RES


@pytest.mark.parametrize("name", list(SHAPES))
def test_direction_residual_default_options(P, name):
    """With the default regularised factor and refine_tol = 1e-10 the returned
    direction solves the unregularised Newton system to 1e-10."""
    lp = _make(name, seed=11)
    A, x, z, rd, rp, rc = _point(lp, 12)
    prob = P.arrowhead_lp_create(lp)
    P.kkt_factor(prob, x, z)
    (dx, dy, dz), info = P.kkt_solve(prob, rd, rp, rc)
    assert onewton.relative_residual(A, x, z, dx, dy, dz, rd, rp, rc) < TOL_RES
    assert abs(info["rel_residual"] -
               onewton.relative_residual(A, x, z, dx, dy, dz, rd, rp, rc)) < 1e-11


@pytest.mark.parametrize("name", ["c0", "ragged_tiles", "wide_border"])
def test_adjoint_matches_oracle(P, name):
    lp = _make(name, seed=3)
    A, x, z, gx, gy, gz = _point(lp, 4)
    prob = P.arrowhead_lp_create(lp, _tight(P))
    P.kkt_factor(prob, x, z)
    (lx, ly, lz), info = P.kkt_adjoint_solve(prob, gx, gy, gz)
    ex, ey, ez = oadj.adjoint_dense(A, x, z, gx, gy, gz)
    assert _rel(lx, ex) < TOL_DIR
    assert _rel(ly, ey) < TOL_DIR
    assert _rel(lz, ez) < TOL_DIR


def test_repeat_is_bitwise_deterministic(P):
    lp = _make("ragged_tiles", seed=5)
    A, x, z, rd, rp, rc = _point(lp, 6)
    prob = P.arrowhead_lp_create(lp)
    outs = []
    for _ in range(2):
        P.kkt_factor(prob, x, z)
        (dx, dy, dz), _ = P.kkt_solve(prob, rd, rp, rc)
        outs.append(np.concatenate([dx, dy, dz]))
    assert np.array_equal(outs[0], outs[1])


def test_device_pointers_with_torch(P):
    import torch
    lp = _make("c0", seed=7)
    A, x, z, rd, rp, rc = _point(lp, 8)
    prob = P.arrowhead_lp_create(lp)
    dev = torch.device("cuda:0")
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=dev)  # noqa: E731
    P.kkt_factor(prob, t(x), t(z))
    (dx, dy, dz), _ = P.kkt_solve(prob, t(rd), t(rp), t(rc))
    assert dx.is_cuda
    ex, ey, ez = onewton.direction_dense(A, x, z, rd, rp, rc)
    assert _rel(dx.cpu().numpy(), ex) < TOL_DIR
    assert _rel(dy.cpu().numpy(), ey) < TOL_DIR


def test_errors(P):
    lp = _make("c0")
    prob = P.arrowhead_lp_create(lp)
    n, m = prob.n, prob.m
    with pytest.raises(P.AHLPError) as e:
        P.kkt_solve(prob, np.zeros(n), np.zeros(m), np.zeros(n))
    assert e.value.status == -1
    x = np.ones(n)
    x[3] = -1.0
    with pytest.raises(P.AHLPError) as e:
        P.kkt_factor(prob, x, np.ones(n))
    assert e.value.status == -1


@pytest.mark.parametrize("seed", [0, 4, 9])
def test_shared_iterates_of_oracle_trajectory(P, seed):
    """At the oracle IPM's own iterates (mu >= 1e-6) and with its predictor
    right-hand side, the decomposed solve leaves a Newton residual < 1e-10."""
    from oracle import ipm as oipm
    lp = config0(seed)
    A, b, c = olp.assemble(lp)
    rec = []
    oipm.solve(A, b, c, record=rec)
    prob = P.arrowhead_lp_create(lp, _tight(P))
    checked = 0
    for r in rec:
        if r["mu"] < 1e-6:
            break
        x, y, z = r["x"], r["y"], r["z"]
        rp, rd = olp.residuals(A, b, c, x, y, z)
        rc = -x * z
        P.kkt_factor(prob, x, z)
        (dx, dy, dz), info = P.kkt_solve(prob, rd, rp, rc)
        assert onewton.relative_residual(A, x, z, dx, dy, dz, rd, rp, rc) < TOL_RES
        # forward error: both sides carry about cond(J) * eps of rounding
        J = onewton.newton_matrix_dense(A, x, z)
        bound = max(1e-10, 1e-13 * np.linalg.cond(J))
        ex, ey, ez = onewton.direction_dense(A, x, z, rd, rp, rc)
        got = np.concatenate([dx, dy, dz])
        ref = np.concatenate([ex, ey, ez])
        assert _rel(got, ref) < bound
        checked += 1
    assert checked >= 4
