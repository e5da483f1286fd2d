"""Seeded generators for block-structured (arrowhead) LPs with local linking.

The problem class is the one of Sec. 3.2 (eq. fig:blockstructure) restricted to
equality rows and x >= 0, with the linking rows split into local (two-link) and
global rows as in Sec. 3.3:

    min  c_0' x_0 + sum_i c_i' x_i
    s.t. W_i x_0 + A_i x_i                       = b_i        i = 1..N
         F0_j x_0 + FL_j x_j + FR_j x_{j+1}      = blink_j    j = 1..N-1
         Fg0 x_0 + sum_i Fg_i x_i                = bg
         x >= 0

Naming bridge to the paper: A_i here is the paper's B_i, W_i the paper's A_i,
FL_j / FR_j / F0_j the paper's local link blocks (unprimed, primed, 0-column),
Fg_i its global link rows.

Global orderings used everywhere in this project:
    x = [x_1 .. x_N, x_0]
    y = [y_1 .. y_N, y_link(pair 1..N-1), y_g]
and z is ordered like x.

Everything here is data generation: random sparse patterns and values, plus
the planted right-hand sides b = A x*, c = A' y* + z* that define a planted LP.
Nothing here belongs to the interior-point method.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import structural_rank


@dataclass
class BlockLP:
    N: int
    n0: int
    mg: int
    A: List[sp.csc_matrix]          # N, m_i x n_i
    W: List[sp.csc_matrix]          # N, m_i x n0
    b: List[np.ndarray]             # N, m_i
    c: List[np.ndarray]             # N, n_i
    c0: np.ndarray                  # n0
    l: np.ndarray                   # N-1 local link row counts
    FL: List[sp.csc_matrix]         # N-1, l_j x n_j
    FR: List[sp.csc_matrix]         # N-1, l_j x n_{j+1}
    F0: List[sp.csc_matrix]         # N-1, l_j x n0
    blink: List[np.ndarray]         # N-1, l_j
    Fg: List[sp.csc_matrix]         # N, mg x n_i
    Fg0: sp.csc_matrix              # mg x n0
    bg: np.ndarray                  # mg
    name: str = ""
    xstar: Optional[np.ndarray] = None   # planted primal optimum (global order)
    ystar: Optional[np.ndarray] = None
    zstar: Optional[np.ndarray] = None
    basis: Optional[np.ndarray] = None   # planted basis (nondegenerate plant only)
    meta: dict = field(default_factory=dict)
    # the full statement of Sec. 3.2 (all optional): bounds lb <= x <= ub per
    # block and for x_0, and inequality rows d <= row x <= f of three kinds --
    # block rows D_i x_i + C_i x_0, local link rows GL_j x_j + GR_j x_{j+1}
    # + G0_j x_0 and global rows sum_i Gg_i x_i + Gg0 x_0
    lb: Optional[List[np.ndarray]] = None
    ub: Optional[List[np.ndarray]] = None
    lb0: Optional[np.ndarray] = None
    ub0: Optional[np.ndarray] = None
    D: Optional[List[sp.csc_matrix]] = None
    C: Optional[List[sp.csc_matrix]] = None
    dlo: Optional[List[np.ndarray]] = None
    dhi: Optional[List[np.ndarray]] = None
    GL: Optional[List[sp.csc_matrix]] = None
    GR: Optional[List[sp.csc_matrix]] = None
    G0: Optional[List[sp.csc_matrix]] = None
    glo: Optional[List[np.ndarray]] = None
    ghi: Optional[List[np.ndarray]] = None
    Gg: Optional[List[sp.csc_matrix]] = None
    Gg0: Optional[sp.csc_matrix] = None
    gglo: Optional[np.ndarray] = None
    gghi: Optional[np.ndarray] = None

    # ---- sizes ---------------------------------------------------------
    @property
    def m_sizes(self) -> np.ndarray:
        return np.array([a.shape[0] for a in self.A], dtype=np.int64)

    @property
    def n_sizes(self) -> np.ndarray:
        return np.array([a.shape[1] for a in self.A], dtype=np.int64)

    @property
    def n_total(self) -> int:
        return int(self.n_sizes.sum()) + self.n0

    @property
    def m_total(self) -> int:
        return int(self.m_sizes.sum()) + int(np.sum(self.l)) + self.mg

    def x_offsets(self) -> np.ndarray:
        """Start of x_i in the global x (length N+1; entry N is x_0's start)."""
        return np.concatenate([[0], np.cumsum(self.n_sizes)]).astype(np.int64)

    def y_offsets(self) -> np.ndarray:
        """Start of y_i (i<N), then of the link block (N), then of y_g (N+1)."""
        mo = np.concatenate([[0], np.cumsum(self.m_sizes)])
        return np.concatenate([mo, [mo[-1] + int(np.sum(self.l))]]).astype(np.int64)

    def link_offsets(self) -> np.ndarray:
        """Start of each pair's rows inside the link block (length N)."""
        return np.concatenate([[0], np.cumsum(self.l)]).astype(np.int64)

    def c_global(self) -> np.ndarray:
        return np.concatenate(list(self.c) + [self.c0])

    def b_global(self) -> np.ndarray:
        return np.concatenate(list(self.b) + list(self.blink) + [self.bg])


# ---------------------------------------------------------------------------
# random sparse building blocks
# ---------------------------------------------------------------------------

def _distinct_rows(rng: np.random.Generator, m: int, n: int, k: int) -> np.ndarray:
    """(n, k) row indices, distinct within each column, sorted."""
    k = min(k, m)
    if k == 0:
        return np.zeros((n, 0), dtype=np.int64)
    if 2 * k > m:
        # dense-ish: take a random permutation prefix per column
        return np.sort(np.argsort(rng.random((n, m)), axis=1)[:, :k], axis=1)
    rows = rng.integers(0, m, size=(n, k))
    while True:
        rows.sort(axis=1)
        dup = np.zeros_like(rows, dtype=bool)
        dup[:, 1:] = rows[:, 1:] == rows[:, :-1]
        nd = int(dup.sum())
        if nd == 0:
            return rows
        rows[dup] = rng.integers(0, m, size=nd)


def _random_csc(rng, m, n, k_per_col, values="normal") -> sp.csc_matrix:
    rows = _distinct_rows(rng, m, n, k_per_col)
    k = rows.shape[1]
    if k == 0:
        return sp.csc_matrix((m, n))
    if values == "normal":
        vals = rng.standard_normal(n * k)
    else:
        vals = values(n * k)
    colptr = np.arange(0, n * k + 1, k, dtype=np.int64)
    return sp.csc_matrix((vals, rows.ravel(), colptr), shape=(m, n))


def _fill_empty_rows(rng, A: sp.csc_matrix) -> sp.csc_matrix:
    """Give every empty row one N(0,1) entry in a random column."""
    A = A.tocsc()
    counts = np.bincount(A.indices, minlength=A.shape[0])
    empty = np.flatnonzero(counts == 0)
    if len(empty) == 0:
        return A
    extra = sp.csc_matrix(
        (rng.standard_normal(len(empty)), (empty, rng.integers(0, A.shape[1], len(empty)))),
        shape=A.shape)
    A = (A + extra).tocsc()
    A.sort_indices()
    return A


def _random_link_rows(rng, l, n_left, n_right, nnz_left, nnz_right):
    """l rows with nnz_left entries in the left block and nnz_right in the right."""
    def part(n, k):
        if l == 0 or n == 0 or k == 0:
            return sp.csc_matrix((l, n))
        cols = _distinct_rows(rng, n, l, k)          # per row: distinct columns
        r = np.repeat(np.arange(l), cols.shape[1])
        return sp.csc_matrix((rng.standard_normal(r.size), (r, cols.ravel())), shape=(l, n))
    return part(n_left, nnz_left), part(n_right, nnz_right)


def _csc(M) -> sp.csc_matrix:
    M = sp.csc_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    return M


# ---------------------------------------------------------------------------
# planting (definition of the LP data from a chosen primal-dual optimum)
# ---------------------------------------------------------------------------

def _apply_A(lp: BlockLP, x: np.ndarray) -> List[np.ndarray]:
    """Row blocks of A x, block by block (data generation only)."""
    xo = lp.x_offsets()
    xs = [x[xo[i]:xo[i + 1]] for i in range(lp.N)]
    x0 = x[xo[lp.N]:]
    out = [lp.A[i] @ xs[i] + lp.W[i] @ x0 for i in range(lp.N)]
    for j in range(lp.N - 1):
        out.append(lp.FL[j] @ xs[j] + lp.FR[j] @ xs[j + 1] + lp.F0[j] @ x0)
    g = lp.Fg0 @ x0
    for i in range(lp.N):
        g = g + lp.Fg[i] @ xs[i]
    out.append(g)
    return out


def _apply_AT(lp: BlockLP, y: np.ndarray) -> np.ndarray:
    yo = lp.y_offsets()
    lo = lp.link_offsets()
    ys = [y[yo[i]:yo[i + 1]] for i in range(lp.N)]
    yl = y[yo[lp.N]:yo[lp.N + 1]]
    yg = y[yo[lp.N + 1]:]
    yL = [yl[lo[j]:lo[j + 1]] for j in range(lp.N - 1)]
    parts = []
    c0 = lp.Fg0.T @ yg
    for i in range(lp.N):
        v = lp.A[i].T @ ys[i] + lp.Fg[i].T @ yg
        if i < lp.N - 1:
            v = v + lp.FL[i].T @ yL[i]
        if i > 0:
            v = v + lp.FR[i - 1].T @ yL[i - 1]
        parts.append(v)
        c0 = c0 + lp.W[i].T @ ys[i]
    for j in range(lp.N - 1):
        c0 = c0 + lp.F0[j].T @ yL[j]
    return np.concatenate(parts + [c0])


def _set_rhs_from_plant(lp: BlockLP, x, y, z):
    rows = _apply_A(lp, x)
    lp.b = rows[:lp.N]
    lp.blink = rows[lp.N:lp.N + lp.N - 1]
    lp.bg = rows[-1]
    cg = _apply_AT(lp, y) + z
    xo = lp.x_offsets()
    lp.c = [cg[xo[i]:xo[i + 1]].copy() for i in range(lp.N)]
    lp.c0 = cg[xo[lp.N]:].copy()
    lp.xstar, lp.ystar, lp.zstar = x, y, z


def plant_half_zero(lp: BlockLP, rng: np.random.Generator, zero_frac: float = 0.5):
    """x*, z* ~ U(0.1, 1) on a strict complementary split, y* ~ N(0, 1)."""
    n = lp.n_total
    perm = rng.permutation(n)
    nz = int(round(zero_frac * n))
    x = rng.uniform(0.1, 1.0, n)
    z = rng.uniform(0.1, 1.0, n)
    x[perm[:nz]] = 0.0
    z[perm[nz:]] = 0.0
    y = rng.standard_normal(lp.m_total)
    _set_rhs_from_plant(lp, x, y, z)


# ---------------------------------------------------------------------------
# generic random arrowhead LP
# ---------------------------------------------------------------------------

def random_block_lp(seed: int, N: int, m_sizes, n_sizes, nnz_per_col: int, n0: int,
                    w_density: float, l, link_nnz=(5, 5), mg: int = 0,
                    global_nnz: int = 4, x0_link_nnz: int = 0, x0_global_nnz: int = 0,
                    plant: Optional[str] = "half_zero", name: str = "") -> BlockLP:
    """Random arrowhead LP.

    m_sizes/n_sizes: per-block sizes.  nnz_per_col: nonzeros per column of A_i,
    N(0,1) values.  n0 linking columns; each W_i column has round(w_density*m_i)
    N(0,1) entries (w_density = 1 gives dense columns).  l: local link rows per
    adjacent pair (int or array of N-1); each link row has link_nnz[0] entries in
    the left block and link_nnz[1] in the right one.  mg global rows with
    global_nnz entries per block.  plant: "half_zero", "nondegenerate" (small
    instances: dense basis check), "basis_blocks" (large instances) or None.
    """
    rng = np.random.default_rng(seed)
    m_sizes = np.asarray(m_sizes, dtype=np.int64)
    n_sizes = np.asarray(n_sizes, dtype=np.int64)
    if np.isscalar(l) or np.ndim(l) == 0:
        l = np.full(max(N - 1, 0), int(l), dtype=np.int64)
    l = np.asarray(l, dtype=np.int64)
    A, W, Fg = [], [], []
    for i in range(N):
        m, n = int(m_sizes[i]), int(n_sizes[i])
        Ai = _fill_empty_rows(rng, _random_csc(rng, m, n, nnz_per_col))
        if m <= 400:
            # small blocks: insist on numerical full row rank
            while np.linalg.matrix_rank(Ai.toarray()) < m:
                Ai = _fill_empty_rows(rng, _random_csc(rng, m, n, nnz_per_col))
        else:
            while structural_rank(Ai) < m:
                Ai = _fill_empty_rows(rng, _random_csc(rng, m, n, nnz_per_col))
        A.append(_csc(Ai))
        kw = int(round(w_density * m))
        W.append(_csc(_random_csc(rng, m, n0, kw)))
        if mg > 0:
            cols = _distinct_rows(rng, n, mg, global_nnz)
            r = np.repeat(np.arange(mg), cols.shape[1])
            Fg.append(_csc(sp.csc_matrix((rng.standard_normal(r.size), (r, cols.ravel())),
                                         shape=(mg, n))))
        else:
            Fg.append(sp.csc_matrix((0, n)))
    FL, FR, F0 = [], [], []
    for j in range(N - 1):
        a, b = _random_link_rows(rng, int(l[j]), int(n_sizes[j]), int(n_sizes[j + 1]),
                                 link_nnz[0], link_nnz[1])
        FL.append(_csc(a))
        FR.append(_csc(b))
        if x0_link_nnz > 0 and n0 > 0 and l[j] > 0:
            f0, _ = _random_link_rows(rng, int(l[j]), n0, 0, min(x0_link_nnz, n0), 0)
            F0.append(_csc(f0))
        else:
            F0.append(sp.csc_matrix((int(l[j]), n0)))
    if mg > 0 and x0_global_nnz > 0 and n0 > 0:
        g0, _ = _random_link_rows(rng, mg, n0, 0, min(x0_global_nnz, n0), 0)
        Fg0 = _csc(g0)
    else:
        Fg0 = sp.csc_matrix((mg, n0))
    lp = BlockLP(N=N, n0=n0, mg=mg, A=A, W=W, b=[], c=[], c0=np.zeros(n0), l=l,
                 FL=FL, FR=FR, F0=F0, blink=[], Fg=Fg, Fg0=Fg0, bg=np.zeros(mg), name=name)
    if plant == "half_zero":
        plant_half_zero(lp, rng)
    elif plant == "nondegenerate":
        plant_nondegenerate(lp, rng)
    elif plant == "basis_blocks":
        plant_basis_blocks(lp, rng)
    elif plant is None:
        pass
    else:
        raise ValueError(plant)
    lp.meta.update(seed=seed, nnz_per_col=nnz_per_col, w_density=w_density,
                   link_nnz=tuple(link_nnz), plant=plant)
    return lp


def plant_nondegenerate(lp: BlockLP, rng: np.random.Generator):
    """Nondegenerate plant: |supp x*| = m exactly with A_B nonsingular.

    The basis is drawn at random and redrawn until the dense A_B is well
    conditioned, so this is meant for small instances (adjoint checks).
    x*_B, z*_N ~ U(0.1, 1), y* ~ N(0, 1).
    """
    from scipy.sparse import bmat  # local: assembly only for the rank check
    m, n = lp.m_total, lp.n_total
    Ag = _assemble_for_rank(lp)
    for _ in range(200):
        B = np.sort(rng.choice(n, m, replace=False))
        AB = Ag[:, B].toarray()
        if np.linalg.matrix_rank(AB) == m and np.linalg.cond(AB) < 1e6:
            break
    else:  # pragma: no cover
        raise RuntimeError("no well-conditioned basis found")
    x = np.zeros(n)
    z = rng.uniform(0.1, 1.0, n)
    x[B] = rng.uniform(0.1, 1.0, m)
    z[B] = 0.0
    y = rng.standard_normal(m)
    _set_rhs_from_plant(lp, x, y, z)
    lp.basis = B


def plant_basis_blocks(lp: BlockLP, rng: np.random.Generator):
    """Nondegenerate plant for large block LPs, with a basis built block by block.

    Basic columns: per block i, the m_i columns that a maximum bipartite
    matching of A_i's rows to its randomly permuted columns assigns (so
    A_i[:, B_i] is structurally nonsingular); per local link row and per
    global row, one further column of that row's own support that is not
    basic yet (a random nonbasic column of the blocks it touches if its
    support is used up); the linking variables x_0 stay nonbasic.  So |B| =
    m, A_B has a perfect row-to-column matching, and x*_B, z*_N ~ U(0.1, 1),
    y* ~ N(0, 1) is the unique, strictly complementary optimum whenever A_B
    is numerically nonsingular (tests check it by a sparse LU with a
    condition estimate).
    """
    from scipy.sparse.csgraph import maximum_bipartite_matching
    N = lp.N
    xo = lp.x_offsets()
    n, m = lp.n_total, lp.m_total
    basic = np.zeros(n, dtype=bool)
    for i in range(N):
        mi, ni = lp.A[i].shape
        perm = rng.permutation(ni)
        Ap = sp.csr_matrix(sp.csc_matrix(lp.A[i])[:, perm])
        match = maximum_bipartite_matching(Ap, perm_type="column")   # row -> column
        if np.any(match < 0):
            raise RuntimeError(f"block {i}: A_i has no full row matching")
        basic[xo[i] + perm[match]] = True

    def one_more(cands, blocks):
        cands = [c for c in cands if not basic[c]]
        if not cands:
            cands = [c for b in blocks for c in range(xo[b], xo[b + 1]) if not basic[c]]
        basic[cands[rng.integers(len(cands))]] = True

    for j in range(N - 1):
        FL, FR = sp.csr_matrix(lp.FL[j]), sp.csr_matrix(lp.FR[j])
        for r in range(int(lp.l[j])):
            cands = [xo[j] + int(c) for c in FL[r].indices] + \
                    [xo[j + 1] + int(c) for c in FR[r].indices]
            one_more(cands, (j, j + 1))
    for g in range(lp.mg):
        cands = []
        for i in range(N):
            Fg = sp.csr_matrix(lp.Fg[i])
            cands += [xo[i] + int(c) for c in Fg[g].indices]
        one_more(cands, tuple(range(N)))
    assert int(basic.sum()) == m, (int(basic.sum()), m)
    x = np.zeros(n)
    z = rng.uniform(0.1, 1.0, n)
    x[basic] = rng.uniform(0.1, 1.0, m)
    z[basic] = 0.0
    y = rng.standard_normal(m)
    _set_rhs_from_plant(lp, x, y, z)
    lp.basis = np.flatnonzero(basic)


def _assemble_for_rank(lp: BlockLP) -> sp.csc_matrix:
    """Column-by-column image of the unit vectors (basis drawing only)."""
    n = lp.n_total
    cols = []
    eye = np.eye(n)
    for k in range(n):
        cols.append(np.concatenate(_apply_A(lp, eye[k])))
    return sp.csc_matrix(np.array(cols).T)


# ---------------------------------------------------------------------------
# the five workload shapes
# ---------------------------------------------------------------------------

def config0(seed: int = 0) -> BlockLP:
    """Tiny planted LP: N=4, A_i 40x60 (6 nnz/col), n0=3 dense, l=2 (10 nnz/row)."""
    return random_block_lp(seed, N=4, m_sizes=[40] * 4, n_sizes=[60] * 4, nnz_per_col=6,
                           n0=3, w_density=1.0, l=2, link_nnz=(5, 5), mg=0,
                           name="C0 N=4 40x60 n0=3 l=2")


def config1(seed: int = 1, N: int = 64) -> BlockLP:
    """Uniform blocks: N=64, A_i 2000x3000 (8 nnz/col), n0=50 at 5%, l=20."""
    return random_block_lp(seed, N=N, m_sizes=[2000] * N, n_sizes=[3000] * N, nnz_per_col=8,
                           n0=50, w_density=0.05, l=20, link_nnz=(5, 5), mg=0,
                           name=f"C1 N={N} 2000x3000 n0=50 l=20")


def config2(seed: int = 2, N: int = 512, nondegenerate: bool = False) -> BlockLP:
    """Uneven blocks: m_i ~ U{500..4000}, n_i = floor(1.5 m_i), n0=100 at 5%, l=16.
    nondegenerate: a unique optimal basis built block by block (plant_basis_blocks)
    instead of the half-zero complementary split."""
    rng = np.random.default_rng(seed + 1000)
    m = rng.integers(500, 4001, size=N)
    n = (3 * m) // 2
    return random_block_lp(seed, N=N, m_sizes=m, n_sizes=n, nnz_per_col=8, n0=100,
                           w_density=0.05, l=16, link_nnz=(5, 5), mg=0,
                           plant="basis_blocks" if nondegenerate else "half_zero",
                           name=f"C2 N={N} uneven 500..4000 n0=100 l=16")


def config4(seed: int = 4, N: int = 128):
    """16 independent LPs of the uneven shape with N=128 (seeds seed..seed+15),
    each with a nondegenerate planted optimum (unique optimal basis)."""
    return [config2(seed + k, N=N, nondegenerate=True) for k in range(16)]


def config3(seed: int = 3, days: int = 365, nodes: int = 30, hours: int = 24,
            lines: int = 40, gens: int = 5, n_invest: int = 600,
            planted: bool = False) -> BlockLP:
    """Energy-system-shaped LP: one block per day, hourly steps, storage chain.

    Per hour: rows = node balances (nodes), storage continuity (nodes), line
    limits (lines).  Columns = storage charge/discharge/level (3*nodes), line
    flows (lines), line headroom slacks (lines), generator outputs (gens) and
    load shed per node (nodes, cost 100, keeps the LP feasible).
    Linking variables: n_invest capacity investments; investment k raises the
    limit of line (k mod lines) in every hour of every day.  Local links: the
    storage continuity of hour 0 of day d+1 uses the level of hour 23 of day d
    (nodes rows per pair, so those rows leave the blocks and become two-links).
    One global row caps total generator emissions, with its slack in the last
    day.  Efficiencies U(0.8,1), demands U(0.5,2), costs lognormal(0,1).
    """
    rng = np.random.default_rng(seed)
    H, Nn, L, G = hours, nodes, lines, gens
    # static network: line endpoints, generator nodes, emission factors
    lf = rng.integers(0, Nn, L)
    lt = (lf + 1 + rng.integers(0, Nn - 1, L)) % Nn
    gnode = rng.integers(0, Nn, G)
    emis = rng.uniform(0.5, 1.5, G)
    cap0 = rng.uniform(0.5, 2.0, L)
    inv_line = np.arange(n_invest) % L
    # per-hour column layout
    c_ch, c_dis, c_lev = 0, Nn, 2 * Nn
    c_flow = 3 * Nn
    c_slk = c_flow + L
    c_gen = c_slk + L
    c_shed = c_gen + G
    nh = c_shed + Nn
    # per-hour row layout
    r_bal, r_sto, r_line = 0, Nn, 2 * Nn
    mh = 2 * Nn + L
    A_list, W_list, b_list, c_list, Fg_list = [], [], [], [], []
    FL_list, FR_list = [], []
    gen_cost = rng.lognormal(0.0, 1.0, G)
    inv_cost = rng.lognormal(0.0, 1.0, n_invest) * days * H * 0.01
    for d in range(days):
        rows, cols, vals = [], [], []
        m_d = H * mh
        n_d = H * nh + (1 if d == days - 1 else 0)
        bd = np.zeros(m_d)
        cd = np.zeros(n_d)
        wr, wc, wv = [], [], []
        fgc, fgv = [], []
        for h in range(H):
            ro, co = h * mh, h * nh
            eff_c = rng.uniform(0.8, 1.0, Nn)
            eff_d = rng.uniform(0.8, 1.0, Nn)
            eff_l = rng.uniform(0.8, 1.0, L)
            dem = rng.uniform(0.5, 2.0, Nn)
            for k in range(Nn):
                # balance: gen + discharge - charge + inflow - outflow + shed = demand
                rows += [ro + r_bal + k, ro + r_bal + k]
                cols += [co + c_ch + k, co + c_dis + k]
                vals += [-1.0, eff_d[k]]
                rows.append(ro + r_bal + k); cols.append(co + c_shed + k); vals.append(1.0)
                bd[ro + r_bal + k] = dem[k]
                # storage continuity: level_h - level_{h-1} - eff*charge + discharge = 0
                rows += [ro + r_sto + k, ro + r_sto + k, ro + r_sto + k]
                cols += [co + c_lev + k, co + c_ch + k, co + c_dis + k]
                vals += [1.0, -eff_c[k], 1.0]
                if h > 0:
                    rows.append(ro + r_sto + k); cols.append(co - nh + c_lev + k); vals.append(-1.0)
            for e in range(L):
                rows += [ro + r_bal + lf[e], ro + r_bal + lt[e]]
                cols += [co + c_flow + e, co + c_flow + e]
                vals += [-1.0, eff_l[e]]
                rows += [ro + r_line + e, ro + r_line + e]
                cols += [co + c_flow + e, co + c_slk + e]
                vals += [1.0, 1.0]
                bd[ro + r_line + e] = cap0[e]
            for g in range(G):
                rows.append(ro + r_bal + gnode[g]); cols.append(co + c_gen + g)
                vals.append(rng.uniform(0.8, 1.0))
                fgc.append(co + c_gen + g); fgv.append(emis[g])
            # capacity investments raise line limits: flow + slack - sum kappa*inv = cap0
            for k in range(n_invest):
                wr.append(ro + r_line + inv_line[k]); wc.append(k)
                wv.append(-rng.uniform(0.8, 1.0))
            cd[co + c_ch:co + c_ch + Nn] = 0.01
            cd[co + c_dis:co + c_dis + Nn] = 0.01
            cd[co + c_flow:co + c_flow + L] = 0.01
            cd[co + c_gen:co + c_gen + G] = gen_cost
            cd[co + c_shed:co + c_shed + Nn] = 100.0
        if d == days - 1:
            fgc.append(n_d - 1); fgv.append(1.0)
        A_list.append(_csc(sp.csc_matrix((vals, (rows, cols)), shape=(m_d, n_d))))
        W_list.append(_csc(sp.csc_matrix((wv, (wr, wc)), shape=(m_d, n_invest))))
        Fg_list.append(_csc(sp.csc_matrix((fgv, (np.zeros(len(fgc), dtype=int), fgc)),
                                          shape=(1, n_d))))
        b_list.append(bd)
        c_list.append(cd)
    # two-links: day d+1 hour-0 continuity rows also use day d hour-23 level.
    # Those rows are moved out of block d+1 into the link block of pair d.
    for d in range(days - 1):
        nL = Nn
        A_next = A_list[d + 1].tocsr()
        keep = np.ones(A_next.shape[0], dtype=bool)
        link_rows = np.arange(r_sto, r_sto + Nn)
        keep[link_rows] = False
        FR = A_next[link_rows, :]
        FL = sp.csc_matrix((-np.ones(Nn), (np.arange(Nn), (H - 1) * nh + c_lev + np.arange(Nn))),
                           shape=(nL, A_list[d].shape[1]))
        FL_list.append(_csc(FL))
        FR_list.append(FR)
        A_list[d + 1] = A_next[keep, :]
        W_list[d + 1] = W_list[d + 1].tocsr()[keep, :]
        b_list[d + 1] = np.concatenate([b_list[d + 1][keep], b_list[d + 1][link_rows]])
    # after removing the link rows, fix the stored per-block b and link rhs
    blink = []
    for d in range(days - 1):
        nb = A_list[d + 1].shape[0]
        blink.append(b_list[d + 1][nb:].copy())
        b_list[d + 1] = b_list[d + 1][:nb].copy()
    A_list = [_csc(a) for a in A_list]
    W_list = [_csc(w) for w in W_list]
    FR_list = [_csc(f) for f in FR_list]
    total_gen = days * H * 1.0 * Nn
    lp = BlockLP(N=days, n0=n_invest, mg=1, A=A_list, W=W_list, b=b_list, c=c_list,
                 c0=inv_cost, l=np.full(days - 1, Nn, dtype=np.int64), FL=FL_list,
                 FR=FR_list, F0=[sp.csc_matrix((Nn, n_invest)) for _ in range(days - 1)],
                 blink=blink, Fg=Fg_list, Fg0=sp.csc_matrix((1, n_invest)),
                 bg=np.array([0.6 * total_gen]),
                 name=f"C3 energy {days} days x {H} h x {Nn} nodes"
                      + (" (planted)" if planted else ""))
    if planted:
        plant_half_zero(lp, rng)
    lp.meta.update(seed=seed, planted=planted)
    return lp


def tiny_lp(seed: int, N: int = 2, m: int = 2, n: int = 4, n0: int = 1, l: int = 1,
            mg: int = 0, plant: Optional[str] = "half_zero") -> BlockLP:
    """Tiny arrowhead LP for brute-force checks (m_total <= 8, n_total <= 16)."""
    return random_block_lp(seed, N=N, m_sizes=[m] * N, n_sizes=[n] * N,
                           nnz_per_col=min(2, m), n0=n0, w_density=1.0, l=l,
                           link_nnz=(min(2, n), min(2, n)), mg=mg, global_nnz=min(2, n),
                           x0_link_nnz=1 if n0 else 0, x0_global_nnz=1 if (n0 and mg) else 0,
                           plant=plant, name=f"tiny seed={seed}")


def window(lp: BlockLP, start: int, Np: int) -> BlockLP:
    """The sub-instance made of blocks start .. start+Np-1 and the links
    between them (a contiguous window of the block chain).

    Global rows keep only the window's blocks' entries.  The optimum is
    re-planted (half-zero split) from the restricted data; the result is a
    valid LP of the same shape family, used for bounded timing samples.
    """
    start = max(0, min(start, lp.N - 1))
    Np = max(1, min(Np, lp.N - start))
    e = start + Np
    sub = BlockLP(N=Np, n0=lp.n0, mg=lp.mg, A=lp.A[start:e], W=lp.W[start:e], b=[], c=[],
                  c0=np.zeros(lp.n0), l=np.asarray(lp.l[start:e - 1]), FL=lp.FL[start:e - 1],
                  FR=lp.FR[start:e - 1], F0=lp.F0[start:e - 1], blink=[], Fg=lp.Fg[start:e],
                  Fg0=lp.Fg0, bg=np.zeros(lp.mg),
                  name=f"{lp.name} blocks {start}..{e - 1}")
    rng = np.random.default_rng(12345 + Np + 7919 * start)
    plant_half_zero(sub, rng)
    return sub


def general_block_lp(seed: int, N: int = 4, m: int = 20, n: int = 30, n0: int = 3, l: int = 2,
                     mg: int = 1, mD: int = 4, lG: int = 2, mgG: int = 1) -> BlockLP:
    """An arrowhead LP in the full statement of Sec. 3.2: the equality rows of
    random_block_lp plus block, local-link and global inequality rows, and
    every kind of bound (lower, upper, box, free, fixed) on block and linking
    variables.  A point x~ inside the bounds is drawn first; the equality
    right-hand sides are A x~ and every inequality row holds x~ strictly, so
    the LP is feasible; the objective is a random vector."""
    lp = random_block_lp(seed, N=N, m_sizes=[m] * N, n_sizes=[n] * N, nnz_per_col=3, n0=n0,
                         w_density=0.3, l=l, link_nnz=(2, 2), mg=mg, global_nnz=4,
                         x0_link_nnz=1 if n0 else 0, x0_global_nnz=1 if (n0 and mg) else 0,
                         plant=None, name=f"general seed={seed}")
    rng = np.random.default_rng(seed + 7777)

    def bounds(k):
        x = rng.uniform(-1.0, 1.0, k)
        kind = rng.integers(0, 5, k)   # 0 lower, 1 upper, 2 box, 3 free, 4 lower (often)
        lo = np.where((kind == 0) | (kind == 2) | (kind == 4), x - rng.uniform(0.2, 1, k), -np.inf)
        hi = np.where((kind == 1) | (kind == 2), x + rng.uniform(0.2, 1, k), np.inf)
        fixed = rng.random(k) < 0.05
        lo = np.where(fixed, x, lo)
        hi = np.where(fixed, x, hi)
        return x, lo, hi

    xs, lp.lb, lp.ub = [], [], []
    for _ in range(N):
        x, lo, hi = bounds(n)
        xs.append(x)
        lp.lb.append(lo)
        lp.ub.append(hi)
    x0, lp.lb0, lp.ub0 = bounds(n0)

    def rows(M, k_lo, width):
        """two-sided / one-sided bounds around M x~ for k_lo rows"""
        v = np.asarray(M).ravel()
        kind = rng.integers(0, 3, k_lo)
        lo = np.where(kind >= 1, v - rng.uniform(0.1, width, k_lo), -np.inf)
        hi = np.where(kind != 1, v + rng.uniform(0.1, width, k_lo), np.inf)
        return lo, hi

    lp.D = [_csc(_random_csc(rng, mD, n, 2)) for _ in range(N)]
    lp.C = [_csc(sp.random(mD, n0, density=0.3, random_state=rng,
                           data_rvs=rng.standard_normal)) for _ in range(N)]
    lp.dlo, lp.dhi = [], []
    for i in range(N):
        lo, hi = rows(lp.D[i] @ xs[i] + lp.C[i] @ x0, mD, 1.0)
        lp.dlo.append(lo)
        lp.dhi.append(hi)
    lp.GL = [_csc(sp.random(lG, n, density=0.1, random_state=rng,
                            data_rvs=rng.standard_normal)) for _ in range(N - 1)]
    lp.GR = [_csc(sp.random(lG, n, density=0.1, random_state=rng,
                            data_rvs=rng.standard_normal)) for _ in range(N - 1)]
    lp.G0 = [_csc(sp.random(lG, n0, density=0.3, random_state=rng,
                            data_rvs=rng.standard_normal)) for _ in range(N - 1)]
    lp.glo, lp.ghi = [], []
    for j in range(N - 1):
        lo, hi = rows(lp.GL[j] @ xs[j] + lp.GR[j] @ xs[j + 1] + lp.G0[j] @ x0, lG, 1.0)
        lp.glo.append(lo)
        lp.ghi.append(hi)
    lp.Gg = [_csc(sp.random(mgG, n, density=0.1, random_state=rng,
                            data_rvs=rng.standard_normal)) for _ in range(N)]
    lp.Gg0 = _csc(sp.random(mgG, n0, density=0.5, random_state=rng, data_rvs=rng.standard_normal))
    gx = sum(lp.Gg[i] @ xs[i] for i in range(N)) + lp.Gg0 @ x0
    lp.gglo, lp.gghi = rows(gx, mgG, 2.0)
    # equality right-hand sides through x~, a random objective
    xg = np.concatenate(xs + [x0])
    lp.b = [lp.A[i] @ xs[i] + lp.W[i] @ x0 for i in range(N)]
    lp.blink = [lp.FL[j] @ xs[j] + lp.FR[j] @ xs[j + 1] + lp.F0[j] @ x0 for j in range(N - 1)]
    lp.bg = sum(lp.Fg[i] @ xs[i] for i in range(N)) + lp.Fg0 @ x0 if mg else np.zeros(0)
    lp.c = [rng.standard_normal(n) for _ in range(N)]
    lp.c0 = rng.standard_normal(n0)
    lp.meta.update(x_interior=xg)
    return lp


def prefix(lp: BlockLP, Np: int) -> BlockLP:
    """The sub-instance made of the first Np blocks and their links (see
    window)."""
    sub = window(lp, 0, Np)
    sub.name = f"{lp.name} prefix {min(Np, lp.N)}"
    return sub


CONFIGS = {0: config0, 1: config1, 2: config2, 3: config3, 4: config4}
