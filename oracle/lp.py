"""Monolithic assembly of an arrowhead LP and its optimality measures.

Assembly follows the block statement of Sec. 3.2 (eq. fig:blockstructure,
equality rows only) with the local/global split of the linking rows of Sec. 3.3:
rows [block rows 1..N | local link rows, pair 1..N-1 | global rows], columns
[x_1 .. x_N | x_0].  Optimality measures are those of the KKT conditions of
Sec. 2.2 (eqs. kkt_stationarity, kkt_primal_feasibility, kkt_complementarity).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def assemble(lp):
    """Return (A, b, c) of the monolithic standard-form LP (A in CSR).

    Every block is placed at its (row offset, column offset) in the global
    ordering; nothing is summed, so the result is exactly the block matrix of
    Sec. 3.2/3.3 with the inequality parts dropped.
    """
    N = lp.N
    n_blk = [a.shape[1] for a in lp.A]
    m_blk = [a.shape[0] for a in lp.A]
    col0 = np.concatenate([[0], np.cumsum(n_blk)])            # x_i starts; col0[N] = x_0
    row0 = np.concatenate([[0], np.cumsum(m_blk)])            # y_i starts
    link0 = row0[N] + np.concatenate([[0], np.cumsum(lp.l)])  # pair starts
    g0 = link0[-1]                                            # global rows start
    n = int(col0[N]) + lp.n0
    m = int(g0) + lp.mg
    R, C, V = [], [], []

    def put(Mblk, r, c_):
        Mblk = sp.coo_matrix(Mblk)
        R.append(Mblk.row + r)
        C.append(Mblk.col + c_)
        V.append(Mblk.data)

    for i in range(N):
        put(lp.A[i], row0[i], col0[i])
        put(lp.W[i], row0[i], col0[N])
        put(lp.Fg[i], g0, col0[i])
    for j in range(len(lp.l)):
        put(lp.FL[j], link0[j], col0[j])
        put(lp.FR[j], link0[j], col0[j + 1])
        put(lp.F0[j], link0[j], col0[N])
    put(lp.Fg0, g0, col0[N])
    A = sp.csr_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))),
                      shape=(m, n))
    b = np.concatenate(list(lp.b) + list(lp.blink) + [lp.bg])
    c = np.concatenate(list(lp.c) + [lp.c0])
    assert A.shape == (len(b), len(c))
    return A, b, c


def residuals(A, b, c, x, y, z):
    """Primal residual r_p = b - Ax and dual residual r_d = c - A'y - z."""
    return b - A @ x, c - A.T @ y - z


def measures(A, b, c, x, y, z):
    """Relative infeasibilities, complementarity and gap (Sec. 2.2)."""
    rp, rd = residuals(A, b, c, x, y, z)
    pobj = float(c @ x)
    dobj = float(b @ y)
    return {
        "pinf": float(np.linalg.norm(rp, np.inf) / (1.0 + np.linalg.norm(b, np.inf))),
        "dinf": float(np.linalg.norm(rd, np.inf) / (1.0 + np.linalg.norm(c, np.inf))),
        "mu": float(x @ z / len(x)),
        "pobj": pobj,
        "dobj": dobj,
        "gap": abs(pobj - dobj) / (1.0 + abs(pobj)),
    }
