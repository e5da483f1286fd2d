"""The tile-sparse job table of the tensor-core trailing updates (host logic,
no GPU): ahlp_tile_sparse_jobs, which the first tensor-core factor of a
handle with tile_sparse = 1 builds its per-step job tables with.

Step k of the batched partial Cholesky (the block factorisation and
Schur-contribution steps of Alg. 2) subtracts L_Ik L_Jk' from the trailing
tiles k < J <= I.  Pinned against:
  * the trailing triangle itself: with every tile nonzero the jobs of a step
    cover each trailing lower tile of each block exactly once;
  * a numeric tile-level partial Cholesky (numpy/scipy) of symmetric positive
    definite matrices with the given tile pattern and dense random tiles: a
    job is kept exactly when its product L_(I0, I0+1)k L_Jk' is nonzero, so
    every job that changes a lower tile is kept and no kept job adds only
    zeros to both of its row tiles;
  * the order: the kept jobs are a subsequence of the dense enumeration.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import paper_2412_07731_gb300 as P


def _dense_jobs(T, Tp):
    jobs, _, dense = P.tile_sparse_jobs(T, Tp)
    assert len(jobs) == dense
    return jobs


def _rows_cols(job):
    """Lower tiles (I, J) a job writes."""
    _, I0, J, h = (int(v) for v in job)
    out = [(I0, J)] if J <= I0 else []
    if h:
        out.append((I0 + 1, J))
    return out


@pytest.mark.parametrize("T,Tp", [([1], [1]), ([2], [1]), ([5], [3]), ([6, 3, 9], [6, 2, 7]),
                                  ([8, 8], [8, 0]), ([13, 4, 7, 2], [11, 4, 1, 2])])
def test_dense_jobs_cover_each_trailing_tile_once(T, Tp):
    jobs, off, dense = P.tile_sparse_jobs(T, Tp)
    assert len(jobs) == dense and off[0] == 0 and off[-1] == dense
    assert len(off) == max(Tp) + 1
    for k in range(max(Tp)):
        seen = {}
        for job in jobs[off[k]:off[k + 1]]:
            b = int(job[0])
            assert k < Tp[b]
            for t in _rows_cols(job):
                seen[(b, t)] = seen.get((b, t), 0) + 1
        want = {(b, (I, J)) for b in range(len(T)) if k < Tp[b]
                for I in range(k + 1, T[b]) for J in range(k + 1, I + 1)}
        assert set(seen) == want and all(v == 1 for v in seen.values())
        # blocks in order, each block's jobs contiguous
        bl = [int(j[0]) for j in jobs[off[k]:off[k + 1]]]
        assert bl == sorted(bl)


def _random_pattern(rng, T):
    """Symmetric tile pattern: a band, a few random tiles, the diagonal, and
    dense trailing border rows (like the link and linking-variable rows)."""
    w = int(rng.integers(0, 3))
    nz = np.zeros((T, T), dtype=bool)
    for I in range(T):
        for J in range(max(0, I - w), I + 1):
            nz[I, J] = True
    extra = rng.random((T, T)) < 0.06
    nz |= np.tril(extra)
    nb = int(rng.integers(0, 2))
    if nb:
        nz[T - nb:, :] = True
    nz = nz | nz.T
    np.fill_diagonal(nz, True)
    return nz


def _numeric_tile_factor(rng, nz, Tp, ts=3):
    """Partial Cholesky over the first Tp pivot tiles of an SPD matrix whose
    tiles are dense random where nz is set; returns L's tiles as a dict
    (I, k) -> array for the pivot columns k < Tp, I > k."""
    T = nz.shape[0]
    n = T * ts
    M = np.zeros((n, n))
    for I in range(T):
        for J in range(I + 1):
            if nz[I, J]:
                blk = rng.standard_normal((ts, ts))
                M[I * ts:(I + 1) * ts, J * ts:(J + 1) * ts] = blk
    M = np.tril(M) + np.tril(M, -1).T
    M += np.diag(np.abs(M).sum(axis=1) + 1.0)      # diagonally dominant: SPD
    A = M.copy()
    Lt = {}
    s = lambda i: slice(i * ts, (i + 1) * ts)      # noqa: E731
    for k in range(Tp):
        Lkk = np.linalg.cholesky(A[s(k), s(k)])
        for I in range(k + 1, T):
            Lt[(I, k)] = sla.solve_triangular(Lkk, A[s(I), s(k)].T, lower=True).T
        for I in range(k + 1, T):
            for J in range(k + 1, I + 1):
                A[s(I), s(J)] -= Lt[(I, k)] @ Lt[(J, k)].T
    return Lt


@pytest.mark.parametrize("seed", range(12))
def test_kept_jobs_are_the_nonzero_products(seed):
    rng = np.random.default_rng(seed)
    nblk = int(rng.integers(1, 5))
    T = [int(rng.integers(1, 15)) for _ in range(nblk)]
    Tp = [int(rng.integers(0, t + 1)) for t in T]
    if max(Tp) == 0:
        Tp[0] = T[0]
    pats = [_random_pattern(rng, t) for t in T]
    jobs, off, dense = P.tile_sparse_jobs(T, Tp, pats)
    djobs, doff, _ = P.tile_sparse_jobs(T, Tp)
    assert len(djobs) == dense and len(jobs) <= dense
    Ls = [_numeric_tile_factor(rng, pats[b], Tp[b]) for b in range(nblk)]
    for k in range(max(Tp)):
        kept = [tuple(int(v) for v in j) for j in jobs[off[k]:off[k + 1]]]
        every = [tuple(int(v) for v in j) for j in djobs[doff[k]:doff[k + 1]]]
        # a subsequence of the dense enumeration
        it = iter(every)
        assert all(any(j == e for e in it) for j in kept)
        kset = set(kept)
        for (b, I0, J, h) in every:
            L = Ls[b]
            rows = [L[(I0, k)]] + ([L[(I0 + 1, k)]] if h else [])
            prod = np.vstack(rows) @ L[(J, k)].T
            nonzero = bool(np.any(prod != 0))
            assert ((b, I0, J, h) in kset) == nonzero, (k, b, I0, J, h)
            # the lower tiles it writes: a change there is never skipped
            lower = [prod[:3]] if J <= I0 else []
            if h:
                lower.append(prod[3:])
            if any(np.any(x != 0) for x in lower):
                assert (b, I0, J, h) in kset


def test_the_energy_shaped_band_leaves_most_jobs_out():
    """A long banded block with dense border rows (the shape of a day of the
    energy model: hourly chain, link and linking-variable rows last): most
    jobs drop out."""
    T, w = 40, 1
    nz = np.zeros((T, T), dtype=bool)
    for I in range(T):
        nz[I, max(0, I - w):I + 1] = True
    nz[T - 2:, :] = True
    nz = nz | nz.T
    jobs, _, dense = P.tile_sparse_jobs([T], [T - 2], [nz])
    assert 0 < len(jobs) < 0.25 * dense


def test_invalid_sizes_are_rejected():
    with pytest.raises(P.AHLPError):
        P.tile_sparse_jobs([3], [4])
    with pytest.raises(P.AHLPError):
        P.tile_sparse_jobs([0], [0])
    jobs, off, dense = P.tile_sparse_jobs([], [])
    assert len(jobs) == 0 and dense == 0 and list(off) == [0]
