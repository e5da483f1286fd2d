"""The full LP statement of Sec. 3.2 -- TEST INFRASTRUCTURE ONLY.

    min  c'x
    s.t. A x = b              (equality rows)
         d <= C x <= f        (inequality rows; entries of d may be -inf, of f +inf)
         l <= x <= u          (bounds; entries of l may be -inf, of u +inf)

The oracle reduces it to the standard form of Sec. 2.2 (A' x' = b', x' >= 0)
by the textbook transformations, solves that with ``ipm.solve`` and maps the
solution back:

  * an inequality row becomes the equality C_r x - s_r = 0 with a new
    variable s_r bounded by d_r <= s_r <= f_r;
  * every variable v with bounds (lo, hi), original or slack, is replaced by
        lo finite, hi = +inf :  v = lo + p,               p >= 0
        lo = -inf, hi finite :  v = hi - p,               p >= 0
        both finite          :  v = lo + p, p + w = hi - lo, p, w >= 0
        both infinite        :  v = p - q,                p, q >= 0
    (a fixed variable, lo = hi, takes the box form with hi - lo = 0).

The objective changes by the constant c'(shifts), which ``solve_general`` adds
back.  Plain scipy.sparse and numpy; no blocking or reordering.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import ipm


def to_standard(c, A, b, C, d, f, lo, hi):
    """Standard form of the general LP.  Returns (cs, As, bs, const, back):
    min cs'p s.t. As p = bs, p >= 0 has the optimal value of the general LP
    minus const, and back(p) returns the general LP's x (and the slacks s of
    the inequality rows)."""
    A = sp.csr_matrix(A)
    C = sp.csr_matrix(C) if C is not None else sp.csr_matrix((0, A.shape[1]))
    n = A.shape[1]
    mC = C.shape[0]
    # variables v = [x; s], rows [A x = b; C x - s = 0]
    M = sp.vstack([sp.hstack([A, sp.csr_matrix((A.shape[0], mC))]),
                   sp.hstack([C, -sp.identity(mC, format="csr")])]).tocsc()
    rhs = np.concatenate([np.asarray(b, float), np.zeros(mC)])
    cv = np.concatenate([np.asarray(c, float), np.zeros(mC)])
    lv = np.concatenate([np.asarray(lo, float), np.asarray(d, float)])
    uv = np.concatenate([np.asarray(hi, float), np.asarray(f, float)])
    nv = n + mC
    cols, cost = [], []            # columns of As over p, their costs
    box_rows = []                  # (p index, hi - lo) of boxed variables
    shift = np.zeros(nv)           # v = shift + sum_k sign_k p_k
    recipe = []                    # per v: list of (p index, sign)
    const = 0.0
    for j in range(nv):
        col = M[:, j]
        lj, uj = lv[j], uv[j]
        if np.isfinite(lj):
            shift[j] = lj
            k = len(cols)
            cols.append(col)
            cost.append(cv[j])
            recipe.append([(k, 1.0)])
            if np.isfinite(uj):
                box_rows.append((k, uj - lj))
        elif np.isfinite(uj):
            shift[j] = uj
            k = len(cols)
            cols.append(-col)
            cost.append(-cv[j])
            recipe.append([(k, -1.0)])
        else:
            k = len(cols)
            cols.append(col)
            cols.append(-col)
            cost.extend([cv[j], -cv[j]])
            recipe.append([(k, 1.0), (k + 1, -1.0)])
        const += cv[j] * shift[j]
    # rows for the boxes: p_k + w = hi - lo, with w a new column
    np_ = len(cols)
    m0 = M.shape[0]
    nb = len(box_rows)
    Ap = sp.hstack(cols + [sp.csc_matrix((m0, nb))]).tocsr() if np_ else sp.csr_matrix((m0, nb))
    if nb:
        r = np.arange(nb)
        pk = np.array([k for k, _ in box_rows])
        Bx = sp.csr_matrix((np.ones(2 * nb), (np.concatenate([r, r]),
                                              np.concatenate([pk, np_ + r]))),
                           shape=(nb, np_ + nb))
        As = sp.vstack([Ap, Bx]).tocsr()
        bs = np.concatenate([rhs - M @ shift, np.array([w for _, w in box_rows])])
    else:
        As = Ap.tocsr()
        bs = rhs - M @ shift
    cs = np.concatenate([np.array(cost), np.zeros(nb)])

    def back(p):
        v = shift.copy()
        for j, parts in enumerate(recipe):
            for k, sgn in parts:
                v[j] += sgn * p[k]
        return v[:n], v[n:]

    return cs, As, bs, const, back


def solve_general(c, A, b, C, d, f, lo, hi, tol: float = 1e-9, max_iter: int = 200):
    """Optimum of the general LP: dict(x, s, objective, status, iterations)."""
    cs, As, bs, const, back = to_standard(c, A, b, C, d, f, lo, hi)
    r = ipm.solve(As, bs, cs, tol=tol, max_iter=max_iter)
    x, s = back(r["x"])
    return {"x": x, "s": s, "objective": float(np.dot(c, x)), "status": r["status"],
            "iterations": r["iterations"], "standard_objective": r["pobj"] + const}


def assemble_general(lp):
    """(c, A, b, C, d, f, lo, hi) of an arrowhead LP in the full statement of
    Sec. 3.2, in the global orderings: columns [x_1 .. x_N | x_0], equality rows
    as lp.assemble, inequality rows [block rows of blocks 1..N | local link
    rows of pairs 1..N-1 | global rows].  Missing parts are empty; missing
    bounds are x >= 0."""
    from . import lp as lpm
    A, b, c = lpm.assemble(lp)
    N, n0 = lp.N, lp.n0
    ns = [a.shape[1] for a in lp.A]
    col0 = np.concatenate([[0], np.cumsum(ns)]).astype(int)
    n = int(col0[N]) + n0
    blocks, dl, dh = [], [], []

    def place(parts, nrows):
        R, Cc, V = [], [], []
        for M, c_ in parts:
            if M is None:
                continue
            Mc = sp.coo_matrix(M)
            R.append(Mc.row)
            Cc.append(Mc.col + c_)
            V.append(Mc.data)
        if not R:
            return sp.csr_matrix((nrows, n))
        return sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(Cc))),
                             shape=(nrows, n))

    if getattr(lp, "D", None) is not None:
        for i in range(N):
            blocks.append(place([(lp.D[i], col0[i]),
                                 (lp.C[i] if getattr(lp, "C", None) is not None else None,
                                  col0[N])], lp.D[i].shape[0]))
            dl.append(lp.dlo[i])
            dh.append(lp.dhi[i])
    if getattr(lp, "GL", None) is not None:
        for j in range(N - 1):
            blocks.append(place([(lp.GL[j], col0[j]), (lp.GR[j], col0[j + 1]),
                                 (lp.G0[j] if getattr(lp, "G0", None) is not None else None,
                                  col0[N])], lp.GL[j].shape[0]))
            dl.append(lp.glo[j])
            dh.append(lp.ghi[j])
    if getattr(lp, "Gg", None) is not None and getattr(lp, "gglo", None) is not None:
        mgG = len(lp.gglo)
        blocks.append(place([(lp.Gg[i], col0[i]) for i in range(N)] + [(lp.Gg0, col0[N])], mgG))
        dl.append(lp.gglo)
        dh.append(lp.gghi)
    C = sp.vstack(blocks).tocsr() if blocks else sp.csr_matrix((0, n))
    d = np.concatenate(dl) if dl else np.zeros(0)
    f = np.concatenate(dh) if dh else np.zeros(0)
    lo = np.concatenate([(lp.lb[i] if getattr(lp, "lb", None) is not None else np.zeros(ns[i]))
                         for i in range(N)] +
                        [lp.lb0 if getattr(lp, "lb0", None) is not None else np.zeros(n0)])
    hi = np.concatenate([(lp.ub[i] if getattr(lp, "ub", None) is not None
                          else np.full(ns[i], np.inf)) for i in range(N)] +
                        [lp.ub0 if getattr(lp, "ub0", None) is not None else np.full(n0, np.inf)])
    return c, A, b, C, d, f, lo, hi
