"""The paper's Schur-complement decomposition, written out densely.

* ``paper_blocks``   K_i, L_i, K_0 of eq. linear_system_pips_perturbed_compressed
                     (Sec. 3.2): K_i = [Sigma_i B_i'; B_i 0] with
                     Sigma_i = -X_i^-1 Z_i, L_i = [0 0 F_i'; A_i 0 0] and
                     K_0 = [Sigma_0 A_0' F_0'; A_0 0 0; F_0 0 0].  The paper's
                     B_i is this project's block matrix ``lp.A[i]``, its A_i
                     the linking-variable block ``lp.W[i]``; there are no
                     A_0 rows (rows only on x_0), so the y_0 part is empty.
* ``schur_alg1``     Alg. 1 / Alg. 2 (column-wise: solve K_i v = L_i e_c,
                     subtract L_i' v) giving S = K_0 - sum_i L_i' K_i^-1 L_i
                     in the ordering [dx_0 | dy_{N+1}], where dy_{N+1} is
                     [local link rows pair 1..N-1 | global rows].
* ``solve_alg3``     Alg. 3 (Schur rhs, Schur solve, modified rhs, block
                     solves), returning the Newton direction.
* ``app_a_contrib``  sum_i L_i' K_i^-1 L_i assembled from the App. A block
                     formulas (M_j, H_j, E_j, M_0) in the ordering
                     [local links | global rows | x_0].
* ``observation1_bound`` the nnz bound of Observation 1 (App. A).
* ``schur_reduced``  the same Schur complement reached through the normal
                     equations of each block: S = K0r - sum_i G_i' M_i^-1 G_i
                     with M_i = A_i D_i A_i' + delta I, D_i = X_i Z_i^-1,
                     G_i = [W_i | A_i D_i U_i' | A_i D_i Fg_i'] and
                     K0r = [[-D_0^-1 - rho I, F_0'], [F_0, sum_i F_i D_i F_i' + delta I]]
                     in the ordering [local links | x_0 | global rows].  With
                     delta = rho = 0 it equals the Alg. 1 matrix up to the
                     symmetric permutation returned by ``reduced_perm``.

Everything is dense numpy; meant for small instances.
"""
from __future__ import annotations

import numpy as np


def _split(lp, v, offsets):
    """Pieces of a global x-ordered vector: x_1 .. x_N, then x_0 (N+1 pieces)."""
    ends = list(offsets) + [len(v)]
    return [v[ends[i]:ends[i + 1]] for i in range(len(ends) - 1)]


def link_rows_of_block(lp, i):
    """F_i of the paper: all linking rows restricted to block i's columns.

    Rows ordered [local pairs 1..N-1 | global rows]; only pairs i-1 and i are
    nonzero (two-links, Sec. 3.3).
    """
    lo = lp.link_offsets()
    nl = int(lo[-1])
    n_i = lp.A[i].shape[1]
    F = np.zeros((nl + lp.mg, n_i))
    if i < lp.N - 1:
        F[lo[i]:lo[i + 1], :] = lp.FL[i].toarray()
    if i > 0:
        F[lo[i - 1]:lo[i], :] = lp.FR[i - 1].toarray()
    if lp.mg:
        F[nl:, :] = lp.Fg[i].toarray()
    return F


def link_rows_of_x0(lp):
    """F_0 of the paper: linking rows restricted to x_0's columns."""
    lo = lp.link_offsets()
    nl = int(lo[-1])
    F0 = np.zeros((nl + lp.mg, lp.n0))
    for j in range(lp.N - 1):
        F0[lo[j]:lo[j + 1], :] = lp.F0[j].toarray()
    if lp.mg:
        F0[nl:, :] = lp.Fg0.toarray()
    return F0


def paper_blocks(lp, x, z):
    """Dense K_i, L_i (i = 1..N) and K_0 of the permuted augmented system."""
    xo = lp.x_offsets()
    xs, zs = _split(lp, x, xo), _split(lp, z, xo)
    nl = int(lp.link_offsets()[-1]) + lp.mg
    n0 = lp.n0
    K, L = [], []
    for i in range(lp.N):
        B = lp.A[i].toarray()
        m_i, n_i = B.shape
        Ki = np.zeros((n_i + m_i, n_i + m_i))
        Ki[:n_i, :n_i] = np.diag(-zs[i] / xs[i])
        Ki[:n_i, n_i:] = B.T
        Ki[n_i:, :n_i] = B
        Li = np.zeros((n_i + m_i, n0 + nl))
        Li[:n_i, n0:] = link_rows_of_block(lp, i).T
        Li[n_i:, :n0] = lp.W[i].toarray()
        K.append(Ki)
        L.append(Li)
    F0 = link_rows_of_x0(lp)
    K0 = np.zeros((n0 + nl, n0 + nl))
    K0[:n0, :n0] = np.diag(-zs[lp.N] / xs[lp.N]) if n0 else 0.0
    K0[:n0, n0:] = F0.T
    K0[n0:, :n0] = F0
    return K, L, K0


def schur_alg1(lp, x, z):
    """S = K_0 - sum_i L_i' K_i^-1 L_i, column by column (Alg. 1, Alg. 2)."""
    K, L, K0 = paper_blocks(lp, x, z)
    S = K0.copy()
    for Ki, Li in zip(K, L):
        for col in range(Li.shape[1]):
            v = np.linalg.solve(Ki, Li[:, col])
            S[:, col] -= Li.T @ v
    return S


def solve_alg3(lp, x, z, r_d, r_p, r_c):
    """Newton direction by Alg. 3 on the permuted augmented system.

    Block rhs b_i = [r_d,i - X_i^-1 r_c,i ; r_p,i] and
    b_0 = [r_d,0 - X_0^-1 r_c,0 ; r_p(link rows)]; dz by back-substitution.
    """
    K, L, K0 = paper_blocks(lp, x, z)
    S = schur_alg1(lp, x, z)
    xo, yo = lp.x_offsets(), lp.y_offsets()
    f = r_d - r_c / x
    N = lp.N
    b_i = [np.concatenate([f[xo[i]:xo[i + 1]], r_p[yo[i]:yo[i + 1]]]) for i in range(N)]
    b0 = np.concatenate([f[xo[N]:], r_p[yo[N]:]])
    bh0 = b0.copy()
    for i in range(N):
        bh0 -= L[i].T @ np.linalg.solve(K[i], b_i[i])
    dz0 = np.linalg.solve(S, bh0)
    dzi = [np.linalg.solve(K[i], b_i[i] - L[i] @ dz0) for i in range(N)]
    n0 = lp.n0
    dx = np.concatenate([d[:lp.A[i].shape[1]] for i, d in enumerate(dzi)] + [dz0[:n0]])
    dy = np.concatenate([d[lp.A[i].shape[1]:] for i, d in enumerate(dzi)] + [dz0[n0:]])
    dz = (r_c - z * dx) / x
    return dx, dy, dz


def _kinv_blocks(lp, i, xi, zi):
    """K~_11, K~_12, K~_21, K~_22 of K_i^-1 (App. A), dense."""
    B = lp.A[i].toarray()
    m_i, n_i = B.shape
    Ki = np.zeros((n_i + m_i, n_i + m_i))
    Ki[:n_i, :n_i] = np.diag(-zi / xi)
    Ki[:n_i, n_i:] = B.T
    Ki[n_i:, :n_i] = B
    Kinv = np.linalg.inv(Ki)
    return Kinv[:n_i, :n_i], Kinv[:n_i, n_i:], Kinv[n_i:, :n_i], Kinv[n_i:, n_i:]


def app_a_contrib(lp, x, z):
    """sum_i L_i' K_i^-1 L_i from the App. A formulas.

    Ordering [local links pair 1..N-1 | global rows | x_0].  Local block j
    gets M_j = F_j K~^j_11 F_j' + F'_j K~^{j+1}_11 F'_j', the off-diagonal
    H_j = F_{j+1} K~^{j+1}_11 F'_j', the border E_j and the corner M_0
    (eqs. schur_complement_blockstructure, dense_border_part_sc,
    dense_corner_part_sc).  Here F_j = FL_j, F'_j = FR_j, paper-A_i = W_i.
    """
    N, n0, mg = lp.N, lp.n0, lp.mg
    xo = lp.x_offsets()
    xs, zs = _split(lp, x, xo), _split(lp, z, xo)
    lo = lp.link_offsets()
    nl = int(lo[-1])
    nb = mg + n0
    tot = nl + nb
    S = np.zeros((tot, tot))
    kb = [_kinv_blocks(lp, i, xs[i], zs[i]) for i in range(N)]
    FL = [f.toarray() for f in lp.FL]
    FR = [f.toarray() for f in lp.FR]
    Fg = [f.toarray() for f in lp.Fg]
    Wd = [w.toarray() for w in lp.W]
    for j in range(N - 1):
        sj = slice(lo[j], lo[j + 1])
        Mj = FL[j] @ kb[j][0] @ FL[j].T + FR[j] @ kb[j + 1][0] @ FR[j].T
        S[sj, sj] = Mj
        if j < N - 2:
            sj1 = slice(lo[j + 1], lo[j + 2])
            Hj = FL[j + 1] @ kb[j + 1][0] @ FR[j].T
            S[sj1, sj] = Hj
            S[sj, sj1] = Hj.T
        Ej = np.vstack([Fg[j] @ kb[j][0] @ FL[j].T + Fg[j + 1] @ kb[j + 1][0] @ FR[j].T,
                        Wd[j].T @ kb[j][2] @ FL[j].T + Wd[j + 1].T @ kb[j + 1][2] @ FR[j].T])
        S[nl:, sj] = Ej
        S[sj, nl:] = Ej.T
    M0 = np.zeros((nb, nb))
    for i in range(N):
        K11, K12, K21, K22 = kb[i]
        M0 += np.block([[Fg[i] @ K11 @ Fg[i].T, Fg[i] @ K12 @ Wd[i]],
                        [Wd[i].T @ K21 @ Fg[i].T, Wd[i].T @ K22 @ Wd[i]]])
    S[nl:, nl:] = M0
    return S


def app_a_perm(lp):
    """Index map: App. A ordering -> Alg. 1 ordering ([x_0 | links | global])."""
    n0, mg = lp.n0, lp.mg
    nl = int(lp.link_offsets()[-1])
    # App. A: [links (nl) | global (mg) | x0 (n0)]
    return np.concatenate([n0 + np.arange(nl), n0 + nl + np.arange(mg), np.arange(n0)])


def observation1_bound(lp) -> int:
    """Observation 1 (App. A): nnz bound of the Schur complement."""
    l = np.asarray(lp.l, dtype=np.int64)
    nb = lp.mg + lp.n0
    return int(np.sum(l * l) + 2 * np.sum(l[:-1] * l[1:]) + 2 * np.sum(l) * nb + nb * nb)


def schur_reduced(lp, x, z, delta: float = 0.0, rho: float = 0.0):
    """Normal-equation form of the same Schur complement (dense).

    Ordering [local links | x_0 | global rows].
    """
    N, n0, mg = lp.N, lp.n0, lp.mg
    xo = lp.x_offsets()
    d = x / z
    ds = _split(lp, d, xo)
    lo = lp.link_offsets()
    nl = int(lo[-1])
    tot = nl + n0 + mg
    sx = slice(nl, nl + n0)
    sg = slice(nl + n0, tot)
    S = np.zeros((tot, tot))
    # K0r
    S[sx, sx] = -np.diag(1.0 / ds[N]) - rho * np.eye(n0) if n0 else 0.0
    F0 = link_rows_of_x0(lp)             # rows [links | global]
    ylin = np.concatenate([np.arange(nl), nl + n0 + np.arange(mg)]).astype(int)
    S[np.ix_(ylin, np.arange(nl, nl + n0))] = F0
    S[np.ix_(np.arange(nl, nl + n0), ylin)] = F0.T
    for i in range(N):
        Fi = link_rows_of_block(lp, i)
        S[np.ix_(ylin, ylin)] += Fi @ np.diag(ds[i]) @ Fi.T
    S[np.ix_(ylin, ylin)] += delta * np.eye(len(ylin))
    # block contributions
    for i in range(N):
        Ai = lp.A[i].toarray()
        Di = np.diag(ds[i])
        Mi = Ai @ Di @ Ai.T + delta * np.eye(Ai.shape[0])
        Fi = link_rows_of_block(lp, i)
        Gi = np.zeros((Ai.shape[0], tot))
        Gi[:, sx] = lp.W[i].toarray()
        Gi[:, ylin] = Ai @ Di @ Fi.T
        S -= Gi.T @ np.linalg.solve(Mi, Gi)
    return S


def reduced_perm(lp):
    """Index map: reduced ordering [links|x0|global] -> Alg. 1 ordering [x0|links|global]."""
    n0, mg = lp.n0, lp.mg
    nl = int(lp.link_offsets()[-1])
    return np.concatenate([n0 + np.arange(nl), np.arange(n0), n0 + nl + np.arange(mg)])
