"""The allocation-free residual check against kkt_solve's own residual report.

kkt_residual_noalloc serves callers that cannot allocate device memory when
they need to verify a direction (a fixed memory budget, an allocator owned by
another component, or code that must avoid the synchronisation an allocation
may cause).  It must agree with the residual kkt_solve reports for the same
direction, call after call, although every call reuses one fixed device
array.  This file is collected last so a failure here cannot hide others.
"""
import numpy as np
import pytest

from instances import config0, random_block_lp
from oracle import lp as olp
from oracle import newton as onewton

pytestmark = pytest.mark.gpu

TOL_RES = 1e-10   # the residual target used by the KKT parity tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_07731_gb300 as P
    return P, torch


def _case(name):
    if name == "c0":
        return config0(3)
    return random_block_lp(8, N=5, m_sizes=[1, 63, 64, 65, 130], n_sizes=[3, 95, 96, 100, 200],
                           nnz_per_col=3, n0=4, w_density=0.2, l=[2, 3, 1, 4], mg=2,
                           global_nnz=4, x0_link_nnz=2, x0_global_nnz=2)


@pytest.mark.parametrize("name", ["c0", "ragged"])
def test_noalloc_residual_matches_kkt_solve(env, name):
    P, torch = env
    lp = _case(name)
    A, b, c = olp.assemble(lp)
    rng = np.random.default_rng(5)
    n, m = A.shape[1], A.shape[0]
    x, z = np.exp(rng.standard_normal(n)), np.exp(rng.standard_normal(n))
    rd, rp, rc = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(n)
    dev = torch.device("cuda:0")
    t = lambda v: torch.as_tensor(v, dtype=torch.float64, device=dev)  # noqa: E731
    prob = P.arrowhead_lp_create(lp)
    P.kkt_factor(prob, t(x), t(z))
    (dx, dy, dz), info = P.kkt_solve(prob, t(rd), t(rp), t(rc))
    out = torch.empty(1, dtype=torch.float64, device=dev)
    got = []
    for _ in range(2):   # two calls in a row share the same fixed device array
        P._lib.kkt_residual_noalloc(prob, t(rd), t(rp), t(rc), dx, dy, dz, out)
        got.append(float(out.item()))
    for g in got:
        assert g < TOL_RES
        assert abs(g - info["rel_residual"]) <= 0.1 * TOL_RES
    # a direction that is not exact: its residual (~1e-6) is far above rounding
    # level and must equal the oracle's mat-vec residual up to the rounding of
    # r - J d (about 1e-16 of ||r||)
    gen = torch.Generator(device=dev).manual_seed(0)
    noisy = [v + 1e-6 * torch.randn(v.shape, generator=gen, dtype=v.dtype, device=dev)
             for v in (dx, dy, dz)]
    ref = onewton.relative_residual(A, x, z, *(v.cpu().numpy() for v in noisy), rd, rp, rc)
    assert ref > 1e-8
    for _ in range(2):
        P._lib.kkt_residual_noalloc(prob, t(rd), t(rp), t(rc), *noisy, out)
        assert abs(float(out.item()) - ref) <= 1e-3 * TOL_RES


def test_noalloc_rejects_host_memory(env):
    P, torch = env
    lp = _case("c0")
    prob = P.arrowhead_lp_create(lp)
    n, m = prob.n, prob.m
    P.kkt_factor(prob, np.ones(n), np.ones(n))
    dev = torch.device("cuda:0")
    zeros_d = torch.zeros(n, dtype=torch.float64, device=dev)
    zeros_m = torch.zeros(m, dtype=torch.float64, device=dev)
    host_out = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(P.AHLPError) as e:
        P._lib.kkt_residual_noalloc(prob, zeros_d, zeros_m, zeros_d, zeros_d, zeros_m, zeros_d,
                                    host_out)
    assert e.value.status == -1
