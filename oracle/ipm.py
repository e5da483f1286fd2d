"""Mehrotra predictor-corrector IPM on the monolithic Newton system.

The paper uses an infeasible primal-dual IPM with Mehrotra's predictor-
corrector scheme (Sec. 2, intro; Sec. 2.3) and defers the details to the
literature.  This oracle fills them in with the standard textbook choices:

  * starting point (Mehrotra's heuristic): x~ = A'(AA')^-1 b,
    y~ = (AA')^-1 A c, z~ = c - A'y~; shift x~, z~ by max(-1.5 min, 0); then
    add 0.5 x^'z^/sum(z^) to x and 0.5 x^'z^/sum(x^) to z;
  * residuals r_p = b - Ax, r_d = c - A'y - z, mu = x'z/n;
  * predictor: r_c = -XZe, step lengths by the ratio test capped at 1;
  * centering sigma = (mu_aff / mu)^3;
  * corrector: r_c = sigma mu e - XZe - dX_aff dZ_aff e;
  * separate primal/dual steps alpha = min(1, eta alpha_max), eta = 0.9995;
  * stop when relative primal and dual infeasibility and the relative gap
    are all <= tol (1e-8 by default).

No Gondzio correctors (they are an optional extension in the paper).
"""
from __future__ import annotations

import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import lp as lpm
from . import newton


def max_step(v: np.ndarray, dv: np.ndarray) -> float:
    """Largest alpha in [0, inf) with v + alpha dv >= 0 (ratio test)."""
    neg = dv < 0
    if not np.any(neg):
        return np.inf
    return float(np.min(-v[neg] / dv[neg]))


def starting_point(A, b, c):
    """Mehrotra's heuristic starting point."""
    A = sp.csr_matrix(A)
    AAt = (A @ A.T).tocsc()
    if AAt.shape[0] <= 4000:
        Md = AAt.toarray()
        solve = lambda r: np.linalg.solve(Md, r)  # noqa: E731
    else:
        lu = spla.splu(AAt)
        solve = lu.solve
    x = A.T @ solve(b)
    y = solve(A @ c)
    z = c - A.T @ y
    xh = x + max(-1.5 * float(np.min(x)), 0.0)
    zh = z + max(-1.5 * float(np.min(z)), 0.0)
    xz = float(xh @ zh)
    x = xh + 0.5 * xz / float(np.sum(zh))
    z = zh + 0.5 * xz / float(np.sum(xh))
    return x, y, z


def solve(A, b, c, tol: float = 1e-8, max_iter: int = 200, eta: float = 0.9995,
          x0=None, y0=None, z0=None, dense_limit: int = 4000, verbose: bool = False,
          record=None):
    """Run the IPM.  Returns dict with x, y, z, iterations, status, measures."""
    A = sp.csr_matrix(A)
    m, n = A.shape
    if x0 is None:
        x, y, z = starting_point(A, b, c)
    else:
        x, y, z = np.array(x0, float), np.array(y0, float), np.array(z0, float)
    status = "max_iter"
    t_kkt = 0.0
    it = 0
    for it in range(max_iter + 1):
        r_p, r_d = lpm.residuals(A, b, c, x, y, z)
        meas = lpm.measures(A, b, c, x, y, z)
        if record is not None:
            record.append(dict(meas, iter=it, x=x.copy(), y=y.copy(), z=z.copy()))
        if verbose:
            print(it, meas)
        if meas["pinf"] <= tol and meas["dinf"] <= tol and meas["gap"] <= tol:
            status = "optimal"
            break
        if it == max_iter:
            break
        mu = meas["mu"]
        # predictor
        t0 = time.perf_counter()
        dxa, dya, dza = newton.direction(A, x, z, r_d, r_p, -x * z, dense_limit)
        t_kkt += time.perf_counter() - t0
        ap = min(1.0, max_step(x, dxa))
        ad = min(1.0, max_step(z, dza))
        mu_aff = float((x + ap * dxa) @ (z + ad * dza)) / n
        sigma = (mu_aff / mu) ** 3
        # corrector
        r_c = sigma * mu - x * z - dxa * dza
        t0 = time.perf_counter()
        dx, dy, dz = newton.direction(A, x, z, r_d, r_p, r_c, dense_limit)
        t_kkt += time.perf_counter() - t0
        ap = min(1.0, eta * max_step(x, dx))
        ad = min(1.0, eta * max_step(z, dz))
        x = x + ap * dx
        y = y + ad * dy
        z = z + ad * dz
    meas = lpm.measures(A, b, c, x, y, z)
    return {"x": x, "y": y, "z": z, "iterations": it, "status": status,
            "kkt_seconds": t_kkt, **meas}


def solve_blocklp(lp, **kw):
    A, b, c = lpm.assemble(lp)
    return solve(A, b, c, **kw)
