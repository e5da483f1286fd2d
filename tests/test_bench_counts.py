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
