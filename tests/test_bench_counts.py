"""The algorithmic work bench.py divides by in its rooflines.

block_factor_flops: the flop count of one batched partial Cholesky of the
augmented block matrices, pinned against an explicit count of the divisions
and multiply-adds of a column-by-column partial Cholesky on small blocks
(and checked to give that factorisation, against scipy's Cholesky)."""
import numpy as np
import pytest

import bench
from instances import random_block_lp


def _partial_cholesky_count(M, p):
    """Right-looking partial Cholesky of M over its first p pivots, counting a
    division as 1 flop and a multiply-add as 2 (the square roots not counted)."""
    a = M.shape[0]
    L = np.tril(M.astype(float))
    flops = 0
    for c in range(p):
        L[c, c] = np.sqrt(L[c, c])
        for r in range(c + 1, a):
            L[r, c] /= L[c, c]
            flops += 1
        for r in range(c + 1, a):
            for s in range(c + 1, r + 1):
                L[r, s] -= L[r, c] * L[s, c]
                flops += 2
    return L, flops


@pytest.mark.parametrize("seed", [0, 1])
def test_block_factor_flops_is_the_partial_cholesky_count(seed):
    lp = random_block_lp(seed, N=3, m_sizes=[5, 7, 4], n_sizes=[8, 10, 6], nnz_per_col=2, n0=2,
                         w_density=0.5, l=[2, 3], mg=1, global_nnz=2)
    rng = np.random.default_rng(seed)
    total = 0
    for i, A in enumerate(lp.A):
        m = A.shape[0]
        k = lp.n0 + lp.mg + (int(lp.l[i - 1]) if i > 0 else 0) + (int(lp.l[i]) if i < lp.N - 1 else 0)
        a = m + k
        B = rng.standard_normal((a, a + 3))
        M = B @ B.T + a * np.eye(a)
        L, f = _partial_cholesky_count(M, m)
        np.testing.assert_allclose(np.tril(L[:m, :m]), np.linalg.cholesky(M[:m, :m]), rtol=1e-12)
        total += f
    assert bench.block_factor_flops(lp) == total


def test_block_factor_roofline_uses_the_update_operand_peak():
    """With the trailing updates on the tensor cores the block factor is
    reported against the tensor peak of the updates' operand type (TF32 for
    FP32 factors: 3 split MMAs per product; FP16 digits for float-float: 21),
    and with the FP32-pipe updates against the FP32 pipe."""
    from types import SimpleNamespace
    lp = random_block_lp(3, N=3, m_sizes=[70, 130, 90], n_sizes=[100, 190, 140], nnz_per_col=3,
                         n0=2, w_density=0.5, l=[2, 3], mg=1, global_nnz=2)
    peaks = {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0,
             "source": "test"}
    _, upd = bench.update_geometry(lp)
    for name, key, per, ratio in (("FP32", "fp32", 3, bench.TF32_PER_BF16),
                                  ("float-float", "ff", 21, bench.FP16_PER_BF16)):
        acc = {"factors_fp32": 0, "ms_block_fp32": 0.0, "factors_ff": 0, "ms_block_ff": 0.0,
               "factors_fp64": 0, "ms_block_fp64": 0.0}
        acc[f"factors_{key}"] = 2
        acc[f"ms_block_{key}"] = 4.0   # 2 ms per factor
        win = SimpleNamespace(acc=acc)
        for variant in (0, 2, 3):
            opts = SimpleNamespace(fp32_update=variant, ff_update=variant)
            r = bench.roofline(lp, win, peaks, opts)
            assert r["bound"] == "tensor" and name in r["kernel"]
            assert r["achieved"] == pytest.approx(per * upd / 2e-3 / 1e12)
            assert r["peak"] == pytest.approx(1700.0 * ratio)
            assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
        r = bench.roofline(lp, win, peaks, SimpleNamespace(fp32_update=1, ff_update=1))
        assert r["bound"] == "alu"


def test_update_geometry_is_the_trailing_update_count():
    """update_geometry's flops are the multiply-adds of the column-by-column
    partial Cholesky that land right of the pivot's 64-column tile (the
    trailing updates; the rest belongs to the diagonal tile and the panel),
    and its entries are the trailing lower triangles summed over the steps."""
    lp = random_block_lp(5, N=2, m_sizes=[150, 70], n_sizes=[220, 100], nnz_per_col=3, n0=2,
                         w_density=0.5, l=[3], mg=1, global_nnz=2)
    NB = 64
    elems = flops = 0
    for i, A in enumerate(lp.A):
        m = A.shape[0]
        a = m + lp.n0 + lp.mg + (int(lp.l[i - 1]) if i > 0 else 0) + \
            (int(lp.l[i]) if i < lp.N - 1 else 0)
        for c in range(m):
            lo = NB * (c // NB + 1)   # first column right of c's tile
            for r in range(lo, a):
                flops += 2 * (r - lo + 1)
        for k in range((m + NB - 1) // NB):
            t = a - NB * (k + 1)
            elems += t * (t + 1) // 2 if t > 0 else 0
    assert bench.update_geometry(lp) == (elems, flops)


def test_tile_sparse_jobs_scale_the_roofline_work():
    """When the tile-sparse enumeration leaves tile jobs out, the update's
    algorithmic work is scaled by the kept fraction and the roofline records
    both job counts; with every job kept nothing changes."""
    from types import SimpleNamespace
    lp = random_block_lp(3, N=3, m_sizes=[70, 130, 90], n_sizes=[100, 190, 140], nnz_per_col=3,
                         n0=2, w_density=0.5, l=[2, 3], mg=1, global_nnz=2)
    e, f = bench.update_geometry(lp)
    assert bench.update_geometry(lp, jobs=(10, 10)) == (e, f)
    assert bench.update_geometry(lp, jobs=(0, 0)) == (e, f)
    e4, f4 = bench.update_geometry(lp, jobs=(1, 4))
    assert e4 == pytest.approx(e / 4) and f4 == pytest.approx(f / 4)
    assert bench.tile_sparse_note((10, 10)) is None
    assert bench.tile_sparse_note((1, 4))["jobs_kept"] == 1
    peaks = {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0,
             "source": "test"}
    acc = {"factors_fp32": 2, "ms_block_fp32": 4.0, "factors_ff": 0, "ms_block_ff": 0.0,
           "factors_fp64": 0, "ms_block_fp64": 0.0}
    opts = SimpleNamespace(fp32_update=3, ff_update=3)
    dense = bench.roofline(lp, SimpleNamespace(acc=acc), peaks, opts)
    sparse = bench.roofline(lp, SimpleNamespace(acc=acc), peaks, opts, (1, 4))
    assert "tile_sparse" not in dense and sparse["tile_sparse"]["jobs_dense"] == 4
    assert sparse["achieved"] == pytest.approx(dense["achieved"] / 4)


def test_kernel_roofline_from_recorded_kernel_times():
    """The headline roofline of the trailing-update kernel, from the kernel
    times a factor records (stand-in handle): algorithmic bytes over the
    update's time against the copy bandwidth, no traffic figure for kernel
    code without a capture, and the kept fraction applied when the
    tile-sparse enumeration left jobs out."""
    from types import SimpleNamespace
    import paper_2412_07731_gb300 as P
    lp = random_block_lp(3, N=3, m_sizes=[70, 130, 90], n_sizes=[100, 190, 140], nnz_per_col=3,
                         n0=2, w_density=0.5, l=[2, 3], mg=1, global_nnz=2)
    peaks = {"bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "hbm_gbs": 6800.0,
             "source": "test"}

    class Handle:
        def __init__(self, jobs):
            self.jobs = jobs
            self.PREC_MIXED, self.PREC_FP64 = P.PREC_MIXED, P.PREC_FP64

        def set_options(self, prob, o):
            prob.options = o

        def kkt_factor(self, prob, x, z):
            pass

        def kkt_factor_kernel_times(self, prob):
            return {"update_ms": 2.0, "update_launches": 10, "diag_ms": 0.1, "panel_ms": 0.2}

        def kkt_update_jobs(self, prob):
            return self.jobs

    elems, _ = bench.update_geometry(lp)
    for prec, word, key in (("FP32", 4, ("FP32", 3)), ("float-float", 8, ("float-float", 3))):
        prob = SimpleNamespace(options=P.default_options(fp32_update=3, ff_update=3))
        r = bench.kernel_roofline(Handle((40, 40)), prob, lp, None, None, prec, peaks)
        gbs = 2 * word * elems / 2e-3 / 1e9
        assert r["bound"] == "hbm" and r["achieved"] == pytest.approx(gbs)
        assert r["frac"] == pytest.approx(gbs / 6800.0)
        assert r["traffic"] is None and "tile_sparse" not in r
        last = bench.UPDATE_TRAFFIC_AT_LAST_CAPTURE[key]
        assert r["traffic_at_last_capture"]["bytes"] == pytest.approx(
            last * 2 * word * elems / 10)
        s = bench.kernel_roofline(Handle((10, 40)), prob, lp, None, None, prec, peaks)
        assert s["achieved"] == pytest.approx(gbs / 4) and s["tile_sparse"]["jobs_kept"] == 10
