"""Differentiation of the LP optimum through torch.autograd (LPSolve).

Pins, on nondegenerate planted arrowhead LPs (x*, y*, z* known, the
optimal basis unique):
  * envelope theorem: d(c'x*)/dc = x*, d(c'x*)/db = y*;
  * the vector-Jacobian product solves J' lam = g for the oracle's dense
    Newton matrix at the returned point, and matches the oracle's dense
    adjoint there;
  * central finite differences (h = 1e-6) of g'x*(b) and of c'x*(c).
"""
import numpy as np
import pytest

from instances import random_block_lp
from oracle import adjoint as oadj
from oracle import lp as olp
from oracle.newton import newton_matrix_dense

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _nondegenerate(seed):
    return random_block_lp(seed, N=4, m_sizes=[40] * 4, n_sizes=[60] * 4, nnz_per_col=6, n0=3,
                           w_density=1.0, l=2, link_nnz=(5, 5), mg=0, plant="nondegenerate",
                           name=f"nondegenerate C0-shape seed={seed}")


@pytest.fixture(scope="module")
def P():
    import paper_2412_07731_gb300 as P
    return P


def _setup(P, seed, prec=None, tol=1e-8):
    from paper_2412_07731_gb300.autograd import lp_solve
    lp = _nondegenerate(seed)
    prob = P.arrowhead_lp_create(lp, P.default_options(
        precision=P.PREC_FP64 if prec is None else prec, tol=tol))
    dev = torch.device("cuda", 0)
    c = torch.tensor(lp.c_global(), dtype=torch.float64, device=dev, requires_grad=True)
    b = torch.tensor(lp.b_global(), dtype=torch.float64, device=dev, requires_grad=True)
    return lp, prob, c, b, lp_solve


@pytest.mark.parametrize("seed", [11, 12])
@pytest.mark.parametrize("mixed", [False, True])
def test_objective_gradients_are_the_planted_solution(P, seed, mixed):
    lp, prob, c, b, lp_solve = _setup(P, seed, P.PREC_MIXED if mixed else P.PREC_FP64)
    x, y, z = lp_solve(c, b, prob)
    obj = (c * x).sum()
    obj.backward()
    xs, ys = lp.xstar, lp.ystar
    # the returned point is an IPM iterate at relative gap 1e-8, whose
    # distance to the vertex the gradient inherits: ~1e-7 with FP64 factors;
    # up to ~1e-6 when the last factors are float-float (tolerance 1e-5, the
    # finite-difference agreement asked of the gradients)
    tol = 1e-5 if mixed else 1e-6
    assert np.abs(c.grad.cpu().numpy() - xs).max() <= tol * max(1.0, np.abs(xs).max())
    assert np.abs(b.grad.cpu().numpy() - ys).max() <= tol * max(1.0, np.abs(ys).max())
    prob.close()


@pytest.mark.parametrize("seed", [11, 13])
def test_vjp_solves_the_transposed_newton_system(P, seed):
    lp, prob, c, b, lp_solve = _setup(P, seed)
    x, y, z = lp_solve(c, b, prob)
    rng = np.random.default_rng(seed)
    g = [rng.standard_normal(v.numel()) for v in (x, y, z)]
    gt = [torch.tensor(v, dtype=torch.float64, device=x.device) for v in g]
    loss = sum((gi * vi).sum() for gi, vi in zip(gt, (x, y, z)))
    loss.backward()
    A, _, _ = olp.assemble(lp)
    xh, zh = x.detach().cpu().numpy(), z.detach().cpu().numpy()
    n, m = xh.size, A.shape[0]
    J = newton_matrix_dense(A, xh, zh)
    gc, gb = c.grad.cpu().numpy(), b.grad.cpu().numpy()
    # the same transposed solve called directly (the factor is still the one
    # of the returned point): autograd returns its lam_x and lam_y
    (l1, l2, l3), info = P.kkt_adjoint_solve(prob, *gt)
    l1, l2, l3 = (v.cpu().numpy() for v in (l1, l2, l3))
    assert np.abs(gc - l1).max() <= 1e-12 * max(1.0, np.abs(l1).max())
    assert np.abs(gb - l2).max() <= 1e-12 * max(1.0, np.abs(l2).max())
    lam = np.concatenate([l1, l2, l3])
    rhs = np.concatenate(g)
    assert np.linalg.norm(J.T @ lam - rhs) <= 1e-9 * np.linalg.norm(rhs), info
    ex, ey, _ = oadj.adjoint_dense(A, xh, zh, *g)
    assert np.abs(gc - ex).max() <= 1e-6 * max(1.0, np.abs(ex).max())
    assert np.abs(gb - ey).max() <= 1e-6 * max(1.0, np.abs(ey).max())
    prob.close()


def test_finite_differences(P):
    seed, h = 14, 1e-6
    lp, prob, c, b, lp_solve = _setup(P, seed, tol=1e-12)
    rng = np.random.default_rng(seed)
    g = torch.tensor(rng.standard_normal(c.numel()), dtype=torch.float64, device=c.device)
    x, _, _ = lp_solve(c, b, prob)
    (g * x).sum().backward()
    grad_b = b.grad.cpu().numpy().copy()
    c2 = c.detach().clone().requires_grad_(True)
    x2, _, _ = lp_solve(c2, b.detach(), prob)
    (c2 * x2).sum().backward()
    grad_c = c2.grad.cpu().numpy().copy()

    def loss_b(bb):
        xx, _, _ = lp_solve(c.detach(), bb, prob)
        return float((g * xx).sum())

    def obj_c(cc):
        xx, _, _ = lp_solve(cc, b.detach(), prob)
        return float((cc * xx).sum())

    for k in rng.choice(b.numel(), 4, replace=False):
        e = torch.zeros_like(b.detach())
        e[k] = h
        fd = (loss_b(b.detach() + e) - loss_b(b.detach() - e)) / (2 * h)
        assert abs(fd - grad_b[k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, grad_b[k])
    for k in rng.choice(c.numel(), 4, replace=False):
        e = torch.zeros_like(c.detach())
        e[k] = h
        fd = (obj_c(c.detach() + e) - obj_c(c.detach() - e)) / (2 * h)
        assert abs(fd - grad_c[k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, grad_c[k])
    prob.close()


def test_backward_after_the_handle_was_solved_again(P):
    """Two forwards on one handle (the second with another objective), then
    the first is differentiated: backward must use J' at the first optimum,
    so its gradients equal those of a forward + backward on a fresh handle."""
    lp, prob, c, b, lp_solve = _setup(P, 15)
    rng = np.random.default_rng(15)
    g = torch.tensor(rng.standard_normal(c.numel()), dtype=torch.float64, device=c.device)
    x1, _, _ = lp_solve(c, b, prob)
    c_other = (c.detach() * (1.0 + 0.1 * torch.rand_like(c.detach()))).requires_grad_(True)
    x2, _, _ = lp_solve(c_other, b.detach(), prob)
    (g * x1).sum().backward()
    grad_b = b.grad.cpu().numpy().copy()
    _, fresh, c_f, b_f, _ = _setup(P, 15)
    xf, _, _ = lp_solve(c_f, b_f, fresh)
    (g * xf).sum().backward()
    ref = b_f.grad.cpu().numpy()
    assert np.abs(grad_b - ref).max() <= 1e-7 * max(1.0, np.abs(ref).max())
    prob.close()
    fresh.close()
