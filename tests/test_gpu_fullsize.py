"""Parity at the benchmark's full size: the uneven 512-block workload (1.18 M
augmented rows, seed 2), in the configuration the benchmark times (mixed
precision, autotuned trailing-update kernels, the headline handle's options).

At this size the oracle cannot factor the monolithic system, so the checks are
properties that hold at any size, computed on the CPU from the assembled sparse
LP (scipy, FP64):
  * the direction kkt_solve returns at a seeded interior point leaves a
    relative Newton residual ||J d - r|| / ||r|| below 1e-10 (the refinement
    solves the unregularised system; FP32 block factors precondition it, and
    FP64 block factors solve it to that accuracy without refinement);
  * a complete mixed-precision solve ends with relative infeasibilities and
    gap below 1e-8 when measured on the CPU, and its objective lies within
    1e-8 of the planted optimum's.
"""
import numpy as np
import pytest

from instances import config2
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


@pytest.fixture(scope="module")
def c2():
    lp = config2()
    A, b, c = olp.assemble(lp)
    return lp, A, b, c


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_direction_residual_at_full_size(P, c2, prec):
    lp, A, b, c = c2
    n, m = A.shape[1], A.shape[0]
    rng = np.random.default_rng(0)
    x = np.exp(rng.standard_normal(n))
    z = np.exp(rng.standard_normal(n))
    rd, rp, rc = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n)
    opts = (P.default_options(precision=P.PREC_MIXED, fp32_cond_max=1e300) if prec == "mixed"
            else P.default_options(precision=P.PREC_FP64, refine_max=0))
    prob = P.arrowhead_lp_create(lp, opts)
    if prec == "mixed":
        P.autotune(prob)
    P.kkt_factor(prob, x, z, 0.0, 0.0)
    (dx, dy, dz), info = P.kkt_solve(prob, rd, rp, rc)
    res = onewton.relative_residual(A, x, z, dx, dy, dz, rd, rp, rc)
    assert res < 1e-10, (res, info)
    prob.close()


def test_complete_solve_at_full_size(P, c2):
    lp, A, b, c = c2
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=P.PREC_MIXED, max_correctors=0))
    P.autotune(prob)
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0, r
    meas = olp.measures(A, b, c, x, y, z)
    assert meas["pinf"] <= 1e-8 and meas["dinf"] <= 1e-8 and meas["gap"] <= 1e-8, meas
    obj = float(c @ lp.xstar)
    assert abs(meas["pobj"] - obj) <= 1e-8 * (1 + abs(obj))
    prob.close()
