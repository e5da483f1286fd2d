"""Differentiable LP solve: the optimum (x*, y*, z*) as a function of (c, b).

At a solution w = (x, y, z) of the optimality conditions
    F(w; c, b) = [A'y + z - c ; Ax - b ; XZe] = 0        (Sec. 2.3)
the implicit function theorem gives J dw = [dc; db; 0], J the Newton matrix
[0 A' I; A 0 0; Z 0 X] at w.  A loss L(w) with gradient g = (g_x, g_y, g_z)
therefore has dL/dc = lam_x and dL/db = lam_y, where J' lam = g: one
transposed KKT solve (kkt_adjoint_solve) with the block factors of the final
iterate, refined by FGMRES on the exact J'.  Objective gradients follow from
the explicit term: d(c'x*)/dc = x* + lam_x with g_x = c (for a nondegenerate
optimum dx*/dc = 0, so this is x*), d(c'x*)/db = lam_y (= y*).

The handle keeps the structure (A_i, W_i, link rows); forward replaces c and
b (arrowhead_lp_set_cb), solves, and factors at the returned point.  The
IPM's own last factor is at the iterate before the final step, where D =
XZ^-1 differs from the returned point's by orders of magnitude on the
variables that are converging to zero, so it would precondition J' badly;
backward therefore uses the factor taken at the returned point.  If the
handle has been factored again since (another forward, an ipm_solve or a
kkt_factor on it), backward refactors at its own saved point first.
"""
from __future__ import annotations

import torch

from . import _lib as L

_ADJOINT_TOL = 1e-6   # relative residual above which the transposed solve has stalled


def _factor_chain(prob, x, z):
    """kkt_factor at (x, z), answering a NaN pivot with more regularisation
    (dual delta, primal rho); True on success."""
    for delta, rho in ((-1.0, -1.0), (1e-6, 1e-8), (1e-4, 1e-6)):
        try:
            L.kkt_factor(prob, x, z, delta, rho)
            return True
        except L.AHLPError as e:
            if e.status != -4:   # AHLP_ERR_NOT_SPD
                raise
    return False


def _factor_fp64(prob, x, z):
    """The same chain with FP64 block factors, the handle's options restored."""
    opts = L.Options.from_buffer_copy(prob.options)
    fp64 = L.Options.from_buffer_copy(opts)
    fp64.precision = L.PREC_FP64
    L.set_options(prob, fp64)
    try:
        if not _factor_chain(prob, x, z):
            raise RuntimeError("no usable factor at the returned point")
    finally:
        L.set_options(prob, opts)


def _factor_at_optimum(prob, x, z):
    """Factor at the returned point for the transposed solves of backward.  The
    point is extremely ill-conditioned (complementarity ~ the tolerance); the
    factor only preconditions an FGMRES solve of the exact transposed system,
    so a NaN pivot is answered with more regularisation, then an FP64 factor."""
    if not _factor_chain(prob, x, z):
        _factor_fp64(prob, x, z)


class LPSolve(torch.autograd.Function):
    """(x, y, z) = LPSolve.apply(c, b, prob): optimum of min c'x s.t. Ax = b,
    x >= 0 for the handle's structure.  c: [n], b: [m] float64 tensors (CPU or
    CUDA; the outputs live on the same device).  Backward reuses the factor
    taken at the returned point, or refactors there when the handle has been
    factored again in between."""

    @staticmethod
    def forward(ctx, c, b, prob):
        c, b = c.detach().contiguous(), b.detach().contiguous()
        L.set_cb(prob, c, b)
        f64 = dict(dtype=torch.float64, device=c.device)
        x, y, z = torch.empty(prob.n, **f64), torch.empty(prob.m, **f64), torch.empty(prob.n, **f64)
        L.ipm_solve(prob, out=(x, y, z))
        _factor_at_optimum(prob, x, z)
        ctx.prob = prob
        ctx.factor_gen = prob.factor_gen
        ctx.save_for_backward(x, z)
        return x, y, z

    @staticmethod
    def backward(ctx, gx, gy, gz):
        prob = ctx.prob
        x, z = ctx.saved_tensors
        if prob.factor_gen != ctx.factor_gen:
            # the handle was refactored elsewhere since forward: J' must be
            # the one at this solve's optimum
            _factor_at_optimum(prob, x, z)
            ctx.factor_gen = prob.factor_gen
        zeros_n = torch.zeros_like(x)
        gx = zeros_n if gx is None else gx.contiguous()
        gy = torch.zeros(prob.m, dtype=x.dtype, device=x.device) if gy is None else gy.contiguous()
        gz = zeros_n if gz is None else gz.contiguous()
        (lx, ly, _), info = L.kkt_adjoint_solve(prob, gx, gy, gz)
        if not info["rel_residual"] <= _ADJOINT_TOL:
            # the factor of the final iterate is not a good enough
            # preconditioner (mixed precision at an extreme D): refactor in FP64
            _factor_fp64(prob, x, z)
            (lx, ly, _), info = L.kkt_adjoint_solve(prob, gx, gy, gz)
            if not info["rel_residual"] <= _ADJOINT_TOL:
                raise RuntimeError(f"adjoint KKT solve did not converge: {info}")
        return lx, ly, None


def lp_solve(c, b, prob):
    """Differentiable optimum (x*, y*, z*) of the handle's LP with objective c
    and right-hand side b (see LPSolve)."""
    return LPSolve.apply(c, b, prob)
