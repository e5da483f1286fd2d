"""The full LP statement of Sec. 3.2 through the C ABI: block, local-link and
global inequality rows, and lower / upper / box / free / fixed bounds on
block and linking variables.  arrowhead_lp_create reduces such an LP to the
equality form the solver works on; the recovered original variables must be
feasible for the original LP and reach the oracle's optimal objective (the
oracle reduces the LP with its own code and is pinned to HiGHS)."""
import numpy as np
import pytest

from instances import general_block_lp
from oracle import general as ogen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2412_07731_gb300 as P
    return P


def _check(P, lp, prec):
    c, A, b, C, d, f, lo, hi = ogen.assemble_general(lp)
    ref = ogen.solve_general(c, A, b, C, d, f, lo, hi)
    if ref["status"] != "optimal":
        return False
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=prec))
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0
    xo, off = P.recover(prob, x)
    obj = float(c @ xo)
    assert abs(obj - (r["pobj"] + off)) <= 1e-9 * (1 + abs(obj))
    assert abs(obj - ref["objective"]) <= 1e-7 * (1 + abs(ref["objective"])), (obj, ref["objective"])
    tol = 1e-6
    assert np.all(xo >= lo - tol) and np.all(xo <= hi + tol)
    Cx = C @ xo
    assert np.all(Cx >= d - tol) and np.all(Cx <= f + tol)
    assert np.abs(A @ xo - b).max() <= tol * (1 + np.abs(b).max())
    prob.close()
    return True


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_statement_matches_oracle(P, prec):
    pr = P.PREC_MIXED if prec == "mixed" else P.PREC_FP64
    solved = sum(_check(P, general_block_lp(seed), pr) for seed in range(6))
    assert solved >= 3


def test_full_statement_batch(P):
    """Two LPs in the full statement and one in equality form, one handle."""
    from instances import random_block_lp
    lps = [general_block_lp(s) for s in range(6)]
    refs = []
    for q in lps:
        ref = ogen.solve_general(*ogen.assemble_general(q))
        if ref["status"] == "optimal":
            refs.append((q, ref))
    refs = refs[:2]
    eq = random_block_lp(3, N=4, m_sizes=[20] * 4, n_sizes=[30] * 4, nnz_per_col=3, n0=3,
                         w_density=0.3, l=2, mg=1, global_nnz=4, x0_link_nnz=1, x0_global_nnz=1)
    batch = [refs[0][0], eq, refs[1][0]]
    prob = P.arrowhead_lp_create(batch)
    (x, y, z), r = P.ipm_solve(prob)
    assert r["status"] == 0
    xo, off = P.recover(prob, x)
    # original orderings: blocks of every LP, then every LP's linking variables
    nb = [sum(a.shape[1] for a in q.A) for q in batch]
    n0s = [q.n0 for q in batch]
    b0 = np.concatenate([[0], np.cumsum(nb)])
    x00 = b0[-1] + np.concatenate([[0], np.cumsum(n0s)])
    objs = []
    for k, q in enumerate(batch):
        xk = np.concatenate([xo[b0[k]:b0[k + 1]], xo[x00[k]:x00[k + 1]]])
        objs.append(float(q.c_global() @ xk))
    assert abs(objs[0] - refs[0][1]["objective"]) <= 1e-7 * (1 + abs(objs[0]))
    assert abs(objs[2] - refs[1][1]["objective"]) <= 1e-7 * (1 + abs(objs[2]))
    from oracle import ipm as oipm
    ref_eq = oipm.solve_blocklp(eq)
    assert abs(objs[1] - ref_eq["pobj"]) <= 1e-7 * (1 + abs(ref_eq["pobj"]))
    prob.close()
