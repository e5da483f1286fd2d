"""Benchmark: interior-point iterations per second on one GB300.

Workload (default, --workload c2): the batched uneven-block arrowhead LP, N =
512 blocks with m_i ~ U{500..4000} rows and n_i = 1.5 m_i columns (8 nnz per
column, N(0,1) values), 100 linking variables with 5%-dense columns, 16 local
link rows per adjacent pair, planted optimum (seed 2).  Its block factors run
in mixed precision (FP32, float-float near the optimum) with the FP64 Schur
factor and FP64 Krylov refinement, and the same LP with FP64 block factors is
measured beside it.

One step = one IPM iteration: the KKT factor (formation of the block normal
matrices, the batched partial Cholesky with the Schur contributions, the Schur
assembly and its link-chain/border factor), the predictor and corrector solves
with their Krylov refinement, and the step.  Exactly --steps iterations are
timed after --warmup iterations, with CUDA events on the handle's stream at
iteration boundaries (the library's iteration callback); when a solve
converges inside the window the next solve starts from Mehrotra's point again
and its start-up work is timed too, without counting as a step.  The handle
(upload and symbolic analysis) is created before the timed region.

value      IPM iterations/s in mixed precision, inputs resident in HBM
fp64       the same LP and metric with FP64 block factors, beside it (its own
           warm-up and step counts are stated)
solve      one complete solve per precision (iterations, ms, objective error
           against the planted optimum)
c1         the uniform 64-block LP: complete solves, mixed and FP64
e2e        mixed precision end to end through the C ABI from host memory: one
           step creates the handle from the host LP, solves to 1e-8, copies x,
           y, z to pinned host memory and destroys the handle
roofline   the batched block partial Cholesky in the precision that took the
           most time in the timed window
stages     one KKT factor and one preconditioner application, stage by stage
cpu_baseline  the CPU oracle (monolithic sparse-LU Mehrotra IPM) timed on
           contiguous windows of 1, 2 and 4 blocks of the same LP and
           extrapolated with the growth exponent measured on them

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload c2|c1|c3|c4|c1small|c0]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_TFLOPS = 1.25       # nominal GB300 FP64 rate (profiling recipe's table)
# FP32 FMA rate from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flops
# x 2.07 GHz (the maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
HBM_FALLBACK_GBS = 6800.0     # GB300 copy bandwidth when no measured figure is present
BF16_FALLBACK_TFLOPS = 1900.0
TF32_OVER_BF16 = 1.1 / 2.25   # nominal dense TF32 : BF16 tensor rate on GB300
FF_FP32_OPS_PER_MAC = 12      # FP32 instructions of one double-float multiply-add

METRIC = "IPM iters/s & KKT solve ms at rel. gap 1e-8; mixed vs FP64 GPU path, % peak"


def measured_peaks() -> dict:
    """MEASURED_PEAKS.json beside this file (copy bandwidth, cuBLAS bf16), else
    the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained",
                                                     d["bf16_tflops"])),
                "source": "measured"}
    except (OSError, ValueError, KeyError):
        return {"hbm_gbs": HBM_FALLBACK_GBS, "bf16_tflops": BF16_FALLBACK_TFLOPS,
                "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def workload(name: str):
    """(LP or list of LPs, description, planted objective(s) or None)."""
    from instances import config0, config1, config2, config3, config4
    if name == "c2":
        lp = config2()
        return lp, ("uneven arrowhead LP, N=512 blocks, m_i~U{500..4000}, n_i=1.5 m_i "
                    "(8 nnz/col), n0=100 linking vars (5% dense), l=16 links/pair, planted "
                    "(seed 2)"), planted_objective(lp)
    if name == "c1":
        lp = config1()
        return lp, ("uniform arrowhead LP, N=64 blocks of 2000x3000 (8 nnz/col), n0=50 "
                    "linking vars (5% dense), l=20 links/pair, planted (seed 1)"), \
            planted_objective(lp)
    if name == "c3":
        lp = config3()
        return lp, ("energy-system arrowhead LP, 365 daily blocks of 24 h x 30 nodes "
                    "(~2400x3800), 600 capacity investments, 30 storage links/pair, 1 "
                    "emissions row (seed 3, not planted)"), None
    if name == "c4":
        lps = config4()
        return lps, ("16 independent planted LPs of the uneven shape, N=128 blocks each "
                     "(seeds 4..19), one batched handle"), [planted_objective(q) for q in lps]
    if name == "c1small":
        lp = config1(N=8)
        return lp, "uniform arrowhead LP, N=8 blocks of 2000x3000, n0=50, l=20, planted", \
            planted_objective(lp)
    if name == "c0":
        lp = config0()
        return lp, "tiny arrowhead LP, N=4 blocks of 40x60, n0=3, l=2, planted", \
            planted_objective(lp)
    raise ValueError(name)


def planted_objective(lp):
    import numpy as np
    return float(np.dot(lp.c_global(), lp.xstar)) if lp.xstar is not None else None


def _blocks(lp):
    return lp if isinstance(lp, (list, tuple)) else [lp]


def block_factor_flops(lp) -> float:
    """Algorithmic flops of one batched partial Cholesky: for each block the
    augmented order a = m_i + k_i with m_i pivots; column c costs (a-c-1)
    divides and (a-c-1)(a-c) flops of rank-1 update."""
    tot = 0.0
    for q in _blocks(lp):
        N, n0, mg = q.N, q.n0, q.mg
        l = list(int(v) for v in q.l)
        for i, A in enumerate(q.A):
            m = A.shape[0]
            k = n0 + mg + (l[i - 1] if i > 0 else 0) + (l[i] if i < N - 1 else 0)
            a = m + k
            # sum_{c=0}^{m-1} (r + r(r+1)), r = a-c-1, in closed form
            r_hi, r_lo = a - 1, a - m
            s1 = (r_hi * (r_hi + 1) - (r_lo - 1) * r_lo) / 2.0
            s2 = (r_hi * (r_hi + 1) * (2 * r_hi + 1) - (r_lo - 1) * r_lo * (2 * r_lo - 1)) / 6.0
            tot += 2.0 * s1 + s2
    return tot


def factor_geometry(lp, NB=64):
    """(lower 64x64 tiles, lower-triangle entries) over all augmented matrices."""
    tiles = tri = 0
    for q in _blocks(lp):
        for i, A in enumerate(q.A):
            k = q.n0 + q.mg + (int(q.l[i - 1]) if i > 0 else 0) + \
                (int(q.l[i]) if i < q.N - 1 else 0)
            a = A.shape[0] + k
            t = (a + NB - 1) // NB
            tiles += t * (t + 1) // 2
            tri += a * (a + 1) // 2
    return tiles, tri


def stage_rooflines(P, prob, lp, peaks):
    """Per-stage times of one KKT factor and one preconditioner application
    (the block solves, the Schur solve and the back-substitution, no Krylov
    refinement) at a seeded interior point (x, z = exp(N(0,1)), seed 0), with
    CUDA events inside the library; median of three after one warm-up.  Each
    stage against the bound that limits it:
      form   -- HBM: the FP32 lower tiles written (pattern reads not counted);
      block  -- the FP32 block factor against the TF32 tensor peak when its
                updates run on the tensor cores, else the FP32 FMA rate;
      schur  -- FP64 latency (cyclic-reduction levels); its flops per factor,
                sum_j 2 (7/3) l_j^3 + 2 (N-1) l^2 B + B^3 / 3, are reported as
                an FP64 rate;
      apply  -- HBM: the FP32 block factors read twice (forward and backward
                wavefront solves)."""
    import numpy as np
    import torch
    from paper_2412_07731_gb300 import _lib as L
    rng = np.random.default_rng(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    f64 = dict(dtype=torch.float64, device=dev)
    x = torch.tensor(np.exp(rng.standard_normal(prob.n)), **f64)
    z = torch.tensor(np.exp(rng.standard_normal(prob.n)), **f64)
    rp = torch.tensor(rng.standard_normal(prob.m), **f64)
    zero = torch.zeros(prob.n, **f64)
    saved = L.Options.from_buffer_copy(prob.options)
    once = L.Options.from_buffer_copy(saved)
    once.refine_max = 0
    once.fp32_cond_max = 1e300   # FP32 block factors at this point
    P.set_options(prob, once)
    fac, sol = [], []
    try:
        for _ in range(4):
            P.kkt_factor(prob, x, z)
            fac.append(P.kkt_stage_times(prob))
        for _ in range(4):
            P.kkt_solve(prob, zero, rp, zero)
            sol.append(P.kkt_stage_times(prob)["last_solve_ms"])
    finally:
        P.set_options(prob, saved)
    med = lambda v: statistics.median(v[1:])  # noqa: E731
    form_ms = med([f["form_ms"] for f in fac])
    block_ms = med([f["block_factor_ms"] for f in fac])
    schur_ms = med([f["schur_ms"] for f in fac])
    apply_ms = med(sol)
    tiles, tri = factor_geometry(lp)
    form_bytes = tiles * 64 * 64 * 4
    apply_bytes = 2 * tri * 4
    flops = block_factor_flops(lp)
    gbs = lambda b, ms: b / (ms / 1e3) / 1e9  # noqa: E731
    hbm = peaks["hbm_gbs"]
    if saved.fp32_update in (0, 2, 3):   # TF32 split products on the tensor cores
        _, upd_flops = update_geometry(lp, jobs=P.kkt_update_jobs(prob))
        tpeak = peaks["bf16_tflops_sustained"] * TF32_PER_BF16
        ach = 3 * upd_flops / (block_ms / 1e3) / 1e12
        block_stage = {"ms": block_ms, "bound": "tensor (TF32, 3 MMAs per product)",
                       "flop": flops, "achieved_tflops": ach, "peak_tflops": tpeak,
                       "frac": ach / tpeak,
                       "fp32_equivalent_tflops": flops / (block_ms / 1e3) / 1e12}
    else:
        block_stage = {"ms": block_ms, "bound": "alu (FP32)", "flop": flops,
                       "achieved_tflops": flops / (block_ms / 1e3) / 1e12,
                       "frac": flops / (block_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS}
    return {
        "point": "x, z = exp(N(0,1)) (seed 0); FP32 block factors",
        "form": {"ms": form_ms, "bound": "hbm", "bytes": form_bytes,
                 "achieved_gbs": gbs(form_bytes, form_ms),
                 "frac": gbs(form_bytes, form_ms) / hbm},
        "block_factor": block_stage,
        "schur_factor": dict({"ms": schur_ms, "bound": "FP64 latency, cyclic reduction levels"},
                             **schur_rate(lp, schur_ms)),
        "apply": {"ms": apply_ms, "bound": "hbm", "bytes": apply_bytes,
                  "achieved_gbs": gbs(apply_bytes, apply_ms),
                  "frac": gbs(apply_bytes, apply_ms) / hbm},
        "peaks": {"hbm_gbs": hbm, "fp32_tflops": FP32_PEAK_TFLOPS},
    }


def schur_rate(lp, ms):
    """FP64 flops of one Schur-complement factor (block cyclic reduction of
    the link chain and the dense border): sum over pairs 2 (7/3) l_j^3, plus
    2 (N-1) lmax^2 B for the border columns through the chain, plus B^3 / 3
    for the border factor (B = n0 + mg per LP), as a rate over ms."""
    flops = 0.0
    for q in _blocks(lp):
        ls = [int(v) for v in q.l]
        B = q.n0 + q.mg
        lmax = max(ls) if ls else 0
        flops += sum(2.0 * (7.0 / 3.0) * l ** 3 for l in ls)
        flops += 2.0 * len(ls) * lmax ** 2 * B + B ** 3 / 3.0
    return {"flop": flops, "achieved_gflops": flops / (ms / 1e3) / 1e9 if ms > 0 else None}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# timing exactly K IPM iterations
# ---------------------------------------------------------------------------
_COUNTERS = ("ms_factor", "ms_solve", "refine_steps", "factors_fp32", "factors_ff",
             "factors_fp64", "ms_block_fp32", "ms_block_ff", "ms_block_fp64", "correctors")


def max_over_ranks(dist, x, device=None):
    """The maximum of the float x over the ranks of the process group (x
    itself without one): the job's time is its slowest rank's."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, iterations, ms):
    """Whole-job IPM iterations/s of `world` replicas that each ran
    `iterations` iterations, the slowest in `ms` milliseconds."""
    return world * iterations / (ms / 1e3)


class IterWindow:
    """Times exactly `steps` IPM iterations after `warmup` completed ones,
    across as many solves as it takes.  The library calls back at the start
    of every iteration (after the iterate's measures); the callback at
    iteration it >= 1 marks the end of iteration it - 1.  At the boundary that
    completes the warm-up the stream is synchronised (and the ranks meet) and
    a CUDA event is recorded on the handle's stream; at the boundary that
    completes the last timed iteration the end event is recorded, the stream
    synchronised and the solve told to stop."""

    def __init__(self, P, stream, warmup, steps, dist=None, local=0):
        from paper_2412_07731_gb300 import _lib as L
        import torch
        self.P, self.L, self.torch = P, L, torch
        self.stream, self.warmup, self.steps, self.dist, self.local = \
            stream, warmup, steps, dist, local
        self.done = 0
        self.started = False
        self.finished = False
        self.prev = None
        self.acc = {k: 0.0 for k in _COUNTERS}
        self.launch0 = self.launches = 0
        self.sampler = None
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)
        self.solves_started_in_window = 0
        CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32,
                              ctypes.POINTER(L.Result))
        self.cfunc = CB(self._cb)

    def _start(self):
        self.torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()
            self.torch.cuda.synchronize()
        self.sampler = ClockSampler(self.local)
        self.launch0 = self.P.launch_count()
        self.e0.record(self.stream)
        self.started = True

    def _cb(self, ctx, it, res_p):
        r = res_p.contents
        snap = {k: float(getattr(r, k)) for k in _COUNTERS}
        if it == 0:
            if self.warmup == 0 and not self.started:
                self._start()
            elif self.started:
                self.solves_started_in_window += 1
            self.prev = snap
            return 0
        if self.started:
            for k in _COUNTERS:
                self.acc[k] += snap[k] - self.prev[k]
        self.prev = snap
        self.done += 1
        if self.done == self.warmup and not self.started:
            self._start()
        if self.started and self.done == self.warmup + self.steps:
            self.e1.record(self.stream)
            self.torch.cuda.synchronize()
            self.launches = self.P.launch_count() - self.launch0
            self.finished = True
            return 1
        return 0

    def run(self, prob, out):
        """Solve repeatedly on prob until the window is complete; returns the
        timed milliseconds (max over ranks)."""
        L = self.L
        saved = L.Options.from_buffer_copy(prob.options)
        o = L.Options.from_buffer_copy(saved)
        o.iter_cb = ctypes.cast(self.cfunc, ctypes.c_void_p).value
        L.set_options(prob, o)
        try:
            while not self.finished:
                _, r = self.P.ipm_solve(prob, out=out, check=False)
                if r["status"] not in (0, -11):
                    raise RuntimeError(f"IPM solve failed: {r}")
        finally:
            L.set_options(prob, saved)
        self.clocks = self.sampler.stop()
        return max_over_ranks(self.dist, self.e0.elapsed_time(self.e1), out[0].device)


# ---------------------------------------------------------------------------
# CPU oracle samples
# ---------------------------------------------------------------------------
def _smallest_window(lp, width):
    import numpy as np
    m = lp.m_sizes.astype(float)
    cost = [float(np.sum(m[s:s + width] ** 3)) for s in range(max(1, lp.N - width + 1))]
    return int(np.argmin(cost))


def oracle_iteration_seconds(sub):
    """Seconds of one oracle IPM iteration (predictor + corrector on the
    monolithic system) on the LP sub, from the oracle's starting point."""
    from oracle import ipm, lp as olp
    A, b, c = olp.assemble(sub)
    x, y, z = ipm.starting_point(A, b, c)
    t0 = time.perf_counter()
    ipm.solve(A, b, c, max_iter=1, x0=x, y0=y, z0=z)
    return time.perf_counter() - t0, A.shape[0]


def _threads():
    try:
        from threadpoolctl import threadpool_info
        blas = max((d.get("num_threads", 1) for d in threadpool_info()), default=1)
    except Exception:
        blas = None
    return os.cpu_count(), blas


def cpu_baseline(lp, widths=(1, 2, 4)):
    """The oracle timed on contiguous windows of 1, 2 and 4 blocks (the ones
    with the smallest blocks, so the sample stays within ~20 s), one IPM
    iteration each; the time per iteration grows as rows^e with e fitted on
    the samples, and is extrapolated to the whole LP's rows with that e."""
    import numpy as np
    from instances import window
    q = _blocks(lp)[0]
    start = _smallest_window(q, max(widths))
    pts = []
    for w in widths:
        sec, rows = oracle_iteration_seconds(window(q, start, w))
        pts.append((w, rows, sec))
    lr = np.log([p[1] for p in pts])
    lt = np.log([p[2] for p in pts])
    e = float(np.polyfit(lr, lt, 1)[0])
    rows_full = sum(int(x.m_total) for x in _blocks(lp))
    t_full = pts[-1][2] * (rows_full / pts[-1][1]) ** e
    ncpu, blas = _threads()
    return {"value": 1.0 / t_full, "unit": "IPM iters/s", "cores": 1, "kind": "oracle",
            "host_cpus": ncpu, "blas_threads": blas,
            "sample": (f"one oracle IPM iteration (SuperLU factorisations of the monolithic "
                       f"augmented system, one core) on windows of {widths} consecutive blocks "
                       f"starting at block {start}: "
                       + ", ".join(f"{w} blocks {r} rows {s:.2f} s" for w, r, s in pts)
                       + f"; time ~ rows^{e:.2f} fitted on them, extrapolated to "
                         f"{rows_full} rows"),
            "growth_exponent": e, "samples": [{"blocks": w, "rows": r, "s": s}
                                              for w, r, s in pts]}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands.  Each step is one oracle
    IPM iteration on the 2-block window of the workload with the smallest
    blocks; the warm-up also times the 1-block window, and the per-iteration
    time is extrapolated to the whole LP with the growth exponent of those
    two samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from instances import window
    lp, desc, _ = workload(args.workload)
    q = _blocks(lp)[0]
    start = _smallest_window(q, 2)
    w1, w2 = window(q, start, 1), window(q, start, 2)
    s1, r1 = oracle_iteration_seconds(w1)
    for _ in range(max(0, args.warmup - 1)):
        oracle_iteration_seconds(w2)
    secs = []
    r2 = None
    for _ in range(args.steps):
        s, r2 = oracle_iteration_seconds(w2)
        secs.append(s)
    s2 = statistics.mean(secs)
    e = math.log(s2 / s1) / math.log(r2 / r1)
    rows_full = sum(int(x.m_total) for x in _blocks(lp))
    per_iter = s2 * (rows_full / r2) ** e
    value = 1.0 / per_iter
    ncpu, blas = _threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "IPM iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_iter * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": "IPM iters/s", "cores": 1, "kind": "oracle",
                             "host_cpus": ncpu, "blas_threads": blas,
                             "sample": f"each step: one oracle IPM iteration on blocks "
                                       f"{start}..{start + 1} ({r2} rows, mean {s2:.2f} s); "
                                       f"1-block window {r1} rows {s1:.2f} s; time ~ rows^{e:.2f},"
                                       f" extrapolated to {rows_full} rows"},
            "e2e": {"value": value, "unit": "IPM iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def objective_error(P, prob, x, planted):
    """Relative error of c'x against the planted objective (per LP of a batch:
    the largest)."""
    import numpy as np
    if planted is None:
        return None
    xh = x.detach().cpu().numpy()
    c = prob._c_global
    if isinstance(planted, list):
        errs = []
        for (ix, _), q, pobj in zip(prob._layout, prob._lps, planted):
            errs.append(abs(float(np.dot(q.c_global(), xh[ix])) - pobj) / (1 + abs(pobj)))
        return max(errs)
    return abs(float(np.dot(c, xh)) - planted) / (1 + abs(planted))


def create(P, lp, prec, **opts):
    import numpy as np
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=prec, **opts))
    lps = _blocks(lp)
    prob._lps = lps
    prob._layout = P.batch_layout(lps) if len(lps) > 1 else None
    prob._c_global = lps[0].c_global() if len(lps) == 1 else None
    return prob


def window_summary(win, ms, steps):
    a = win.acc
    it = max(steps, 1)
    return {"ms_per_step": ms / it,
            "kkt_factor_ms": a["ms_factor"] / it,
            "kkt_solve_ms_per_iteration": a["ms_solve"] / it,
            "refine_steps_per_iteration": a["refine_steps"] / it,
            "factors": {"fp32": a["factors_fp32"], "float_float": a["factors_ff"],
                        "fp64": a["factors_fp64"]},
            "block_factor_ms": {
                "fp32": a["ms_block_fp32"] / a["factors_fp32"] if a["factors_fp32"] else None,
                "float_float": a["ms_block_ff"] / a["factors_ff"] if a["factors_ff"] else None,
                "fp64": a["ms_block_fp64"] / a["factors_fp64"] if a["factors_fp64"] else None},
            "solves_restarted_in_window": win.solves_started_in_window,
            "correctors": a["correctors"]}


def full_solve(P, prob, out, planted):
    """One complete solve to rel. gap 1e-8 (its own CUDA-event time)."""
    import torch
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    _, r = P.ipm_solve(prob, out=out, check=False)
    e1.record(stream)
    torch.cuda.synchronize()
    if r["status"] != 0:
        raise RuntimeError(f"IPM solve failed: {r}")
    return {"iterations": r["iterations"], "ms": e0.elapsed_time(e1),
            "rel_gap": r["rel_gap"], "pinf": r["pinf"], "dinf": r["dinf"],
            "objective": r["pobj"],
            "objective_error_vs_planted": objective_error(P, prob, out[0], planted),
            "factors": {"fp32": r["factors_fp32"], "float_float": r["factors_ff"],
                        "fp64": r["factors_fp64"]},
            "refine_steps": r["refine_steps"], "escalations": r["escalations"],
            "ms_factor": r["ms_factor"], "ms_solve": r["ms_solve"]}


def update_geometry(lp, NB=64, jobs=None):
    """(lower-triangle entries the trailing updates read and write, summed over
    the steps; their flops) of one batched partial Cholesky: at step k a block
    with T tiles and Tp pivot tiles updates the lower triangle of its trailing
    (a - 64(k+1))-order matrix with the 64 pivot columns of step k (fewer at
    a ragged last pivot tile).  jobs = (kept, dense) tile jobs of the
    tensor-core updates: when the tile-sparse enumeration leaves jobs out,
    both figures are scaled by the kept fraction (jobs of one workload have
    nearly equal sizes; the triangle's diagonal jobs are smaller)."""
    frac = jobs[0] / jobs[1] if jobs and jobs[1] and jobs[0] < jobs[1] else 1.0
    elems, flops = _update_geometry_dense(lp, NB)
    return elems * frac, flops * frac


def tile_sparse_note(jobs):
    """The roofline's record of the tile-sparse enumeration, or None when
    every tile job ran."""
    if not jobs or not jobs[1] or jobs[0] >= jobs[1]:
        return None
    return {"jobs_kept": jobs[0], "jobs_dense": jobs[1],
            "note": "structurally zero tile products left out; algorithmic bytes and "
                    "flops scaled by the kept fraction"}


def _update_geometry_dense(lp, NB):
    elems = flops = 0.0
    for q in _blocks(lp):
        for i, A in enumerate(q.A):
            kk = q.n0 + q.mg + (int(q.l[i - 1]) if i > 0 else 0) + \
                (int(q.l[i]) if i < q.N - 1 else 0)
            m = A.shape[0]
            a = m + kk
            for k in range((m + NB - 1) // NB):
                t = a - NB * (k + 1)
                if t <= 0:
                    break
                piv = min(NB, m - NB * k)
                e = t * (t + 1) / 2.0
                elems += e
                flops += 2.0 * piv * e
    return elems, flops


# DRAM bytes per algorithmic byte of the trailing-update kernels, keyed by
# (precision, update option), from the ncu captures in profiles/ (uniform
# 8-block workload, whose trailing matrices partly fit L2):
# pchol_update_tc_c1small.md (per-tile TF32), pchol_update_tc2_c1small.md
# (persistent TF32), pchol_update_oz2_c1small.md (persistent digits).  The
# live bench scales them by the bytes of its own launches.  Those captures
# predate the kernels' job-table argument (tile-sparse updates; a dense
# workload passes none and reads no table), so roofline.traffic is null and
# the scaled figure goes to traffic_at_last_capture.  UPDATE_TRAFFIC_PER_BYTE
# holds captures of the current kernel code only.
UPDATE_TRAFFIC_AT_LAST_CAPTURE = {("FP32", 2): 0.68, ("FP32", 3): 0.70,
                                  ("float-float", 3): 0.88}
UPDATE_TRAFFIC_PER_BYTE = {}
UPDATE_KERNEL = {("FP32", 1): "pchol_update_f32_kernel (FP32 pipe)",
                 ("FP32", 2): "pchol_update_tc_kernel (tcgen05, one CTA per tile)",
                 ("FP32", 3): "pchol_update_tc2_kernel (tcgen05, persistent)",
                 ("float-float", 1): "pchol_update_ff8_kernel (double-float, FP32 pipe)",
                 ("float-float", 2): "pchol_update_oz_kernel (tcgen05 digits, one CTA per tile)",
                 ("float-float", 3): "pchol_update_oz2_kernel (tcgen05 digits, persistent)"}


def kernel_roofline(P, prob, lp, x, z, prec_name, peaks):
    """The trailing-update kernel of the block factor in precision prec_name at
    the iterate (x, z) where the timed window ended: CUDA events around its
    launches (option profile_kernels), median of three factors after one
    warm-up.  Its algorithmic bytes are the lower-triangle entries it reads
    and writes (4 bytes each way for FP32, 8 for float-float's two words,
    8 for FP64); for FP64 the bound is the FP64 pipe instead."""
    from paper_2412_07731_gb300 import _lib as L
    saved = L.Options.from_buffer_copy(prob.options)
    o = L.Options.from_buffer_copy(saved)
    o.profile_kernels = 1
    o.refine_max = 0
    if prec_name == "FP32":
        o.precision, o.fp32_cond_max = P.PREC_MIXED, 1e300
    elif prec_name == "float-float":
        o.precision, o.fp32_cond_max = P.PREC_MIXED, 1.0
    else:
        o.precision = P.PREC_FP64
    P.set_options(prob, o)
    times = []
    try:
        for _ in range(4):
            P.kkt_factor(prob, x, z)
            times.append(P.kkt_factor_kernel_times(prob))
    finally:
        P.set_options(prob, saved)
    med = lambda key: statistics.median([t[key] for t in times[1:]])  # noqa: E731
    upd_ms, launches = med("update_ms"), med("update_launches")
    jobs = P.kkt_update_jobs(prob)
    variant = (saved.fp32_update if prec_name == "FP32" else saved.ff_update) or 2
    tensor_upd = prec_name != "FP64" and variant in (2, 3)
    elems, flops = update_geometry(lp, jobs=jobs if tensor_upd else None)
    out = {"kernel": f"trailing update of the {prec_name} block factor: "
                     f"{UPDATE_KERNEL.get((prec_name, variant), 'FP64 pipe')}",
           "launches": launches,
           "ms_per_factor": upd_ms, "diag_ms": med("diag_ms"), "panel_ms": med("panel_ms")}
    if prec_name == "FP64":
        ach = flops / (upd_ms / 1e3) / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                    "flop_per_launch": flops / launches,
                    "peak_source": "nominal GB300 FP64 rate"})
        return out
    word = 4 if prec_name == "FP32" else 8
    bytes_ = 2.0 * word * elems
    gbs = bytes_ / (upd_ms / 1e3) / 1e9
    ratio = UPDATE_TRAFFIC_PER_BYTE.get((prec_name, variant))
    last = UPDATE_TRAFFIC_AT_LAST_CAPTURE.get((prec_name, variant))
    if last and not ratio:
        out["traffic_at_last_capture"] = {
            "bytes": last * bytes_ / launches,
            "note": "ncu DRAM bytes per algorithmic byte of the kernel's previous code "
                    "(before its job-table argument), scaled to this launch"}
    sparse = tile_sparse_note(jobs) if tensor_upd else None
    if sparse:
        out["tile_sparse"] = sparse
    out.update({"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / peaks["hbm_gbs"],
                "traffic": ratio * bytes_ / launches if ratio else None,
                "bytes_per_launch": bytes_ / launches,
                "peak_source": f"{peaks['source']} copy bandwidth (MEASURED_PEAKS.json)",
                "tensor": {"flop_per_factor": flops,
                           "achieved_tflops": flops / (upd_ms / 1e3) / 1e12,
                           "note": "FP32: 3 TF32 MMAs per product (hi*hi, hi*lo, lo*hi); "
                                   "float-float: 21 FP16 digit MMAs per product"}})
    return out


# nominal dense tensor rates relative to BF16 (profiling recipe's table:
# bf16/fp16 2.25, tf32 1.1 PFLOP/s): a contraction's peak is the measured BF16
# peak times this ratio
TF32_PER_BF16 = 1.1 / 2.25
FP16_PER_BF16 = 1.0


def roofline(lp, win, peaks, opts=None, jobs=None):
    """The batched block partial Cholesky in the precision whose factors took
    the most time in the timed window; achieved = its algorithmic flops per
    factor / its mean CUDA-event time per factor.  When its trailing updates
    run on the tensor cores (TF32 hi/lo splits: 3 MMAs per product; FP16
    digits: 21), the factor is reported against the tensor peak of that
    operand type, counting the updates' tensor flops (sustained BF16 peak,
    the factor being timed inside long steps)."""
    a = win.acc
    flops = block_factor_flops(lp)
    kinds = [
        (a["factors_fp32"], a["ms_block_fp32"], "FP32", FP32_PEAK_TFLOPS, "TFLOP/s",
         "FP32 FMA rate from unit counts and the maximum SM clock (80.5 TFLOP/s)"),
        (a["factors_ff"], a["ms_block_ff"], "float-float", FP32_PEAK_TFLOPS / 2.0,
         "T FP32-instr/s",
         "FP32 pipe instruction rate from unit counts and clock (40.3e12 instr/s); a "
         "double-float multiply-add is 12 FP32 instructions"),
        (a["factors_fp64"], a["ms_block_fp64"], "FP64", FP64_PEAK_TFLOPS, "TFLOP/s",
         "nominal GB300 FP64 rate"),
    ]
    cnt, tot, name, peak, unit, src = max(kinds, key=lambda k: k[1] if k[0] else -1.0)
    if not cnt:
        return None
    ms = tot / cnt
    variant = None
    if opts is not None:
        variant = (opts.fp32_update if name == "FP32" else
                   opts.ff_update if name == "float-float" else None)
    if variant in (0, 2, 3):   # tensor-core trailing updates
        _, upd_flops = update_geometry(lp, jobs=jobs)
        per, ratio, op = ((3, TF32_PER_BF16, "TF32") if name == "FP32" else
                          (21, FP16_PER_BF16, "FP16"))
        tpeak = peaks["bf16_tflops_sustained"] * ratio
        achieved = per * upd_flops / (ms / 1e3) / 1e12
        out = {"bound": "tensor", "achieved": achieved, "peak": tpeak, "unit": "TFLOP/s",
               "frac": achieved / tpeak, "traffic": None,
               "kernel": f"batched block partial Cholesky ({name}; diagonal tile, panel, "
                         f"trailing update on the tensor cores as {per} {op} MMAs per "
                         f"product), {flops:.4g} flop per factor, {ms:.2f} ms",
               "peak_source": f"{peaks['source']} sustained BF16 peak x {ratio:.3f} "
                              f"(nominal {op}:BF16 dense ratio)",
               "fp64_equivalent_tflops": flops / (ms / 1e3) / 1e12}
        sparse = tile_sparse_note(jobs)
        if sparse:
            out["tile_sparse"] = sparse
        return out
    if name == "float-float":
        achieved = flops / 2.0 * FF_FP32_OPS_PER_MAC / (ms / 1e3) / 1e12
        extra = {"fp64_equivalent_tflops": flops / (ms / 1e3) / 1e12}
    else:
        achieved = flops / (ms / 1e3) / 1e12
        extra = {}
    return dict({"bound": "alu", "achieved": achieved, "peak": peak, "unit": unit,
                 "frac": achieved / peak, "traffic": None,
                 "kernel": f"batched block partial Cholesky ({name}; diagonal tile, panel, "
                           f"trailing update), {flops:.4g} flop per factor, {ms:.2f} ms",
                 "peak_source": src}, **extra)


def run_ours(args):
    import torch
    import paper_2412_07731_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    peaks = measured_peaks()

    lp, desc, planted = workload(args.workload)
    stream = torch.cuda.current_stream(dev)
    headline = P.PREC_MIXED if args.precision == "mixed" else P.PREC_FP64
    other = P.PREC_FP64 if headline == P.PREC_MIXED else P.PREC_MIXED
    # the timed iteration is the plain predictor-corrector step (one factor,
    # predictor and corrector solves)
    opts = dict(max_correctors=args.correctors)
    f64 = dict(dtype=torch.float64, device=dev)

    tuned = {}

    def arm(prec, warmup, steps):
        prob = create(P, lp, prec, **opts)
        P.load().arrowhead_lp_set_stream(prob.handle, stream.cuda_stream)
        if prec == P.PREC_MIXED and not args.no_autotune:
            # the project's autotuner picks the trailing-update kernels of the
            # FP32 and float-float factors on this LP's blocks (before timing)
            tuned.update(P.autotune(prob))
        out = (torch.empty(prob.n, **f64), torch.empty(prob.m, **f64),
               torch.empty(prob.n, **f64))
        win = IterWindow(P, stream, warmup, steps, dist, local)
        ms = win.run(prob, out)
        win.last_out = tuple(t.clone() for t in out)
        full = full_solve(P, prob, out, planted) if not args.no_full_solve else None
        return prob, win, ms, full

    prob, win, ms, full = arm(headline, args.warmup, args.steps)
    value = replica_value(world, args.steps, ms)
    summ = window_summary(win, ms, args.steps)
    factor_roof = roofline(lp, win, peaks, prob.options, P.kkt_update_jobs(prob))
    roof = None
    if factor_roof is not None and rank == 0:
        # the dominant kernel: the trailing update of the block factor in the
        # precision that took the most time, at the window's last iterate
        name = factor_roof["kernel"].split("(")[1].split(";")[0]
        xw, _, zw = win.last_out
        roof = kernel_roofline(P, prob, lp, xw, zw, name, peaks)
    stages = None
    if rank == 0 and headline == P.PREC_MIXED and not args.no_stages:
        stages = stage_rooflines(P, prob, lp, peaks)
    prob.close()
    del prob

    other_line = None
    if not args.no_compare:
        osteps = min(args.steps, args.other_steps)
        ow = min(args.warmup, 2)
        oprob, owin, oms, ofull = arm(other, ow, osteps)
        other_line = dict({"precision": "FP64" if other == P.PREC_FP64 else "mixed",
                           "value": replica_value(world, osteps, oms), "unit": "IPM iters/s",
                           "steps": osteps, "warmup": ow, "clocks": owin.clocks,
                           "solve": ofull}, **window_summary(owin, oms, osteps))
        oprob.close()
        del oprob

    c1 = None
    if args.workload != "c1" and not args.no_c1:
        c1lp, c1desc, c1planted = workload("c1")
        c1 = {"workload": c1desc}
        for prec, name in ((P.PREC_MIXED, "mixed"), (P.PREC_FP64, "fp64")):
            q = create(P, c1lp, prec, **opts)
            P.load().arrowhead_lp_set_stream(q.handle, stream.cuda_stream)
            tuned1 = P.autotune(q) if prec == P.PREC_MIXED and not args.no_autotune else None
            out = (torch.empty(q.n, **f64), torch.empty(q.m, **f64), torch.empty(q.n, **f64))
            full_solve(P, q, out, c1planted)   # warm-up
            runs = [full_solve(P, q, out, c1planted) for _ in range(2)]
            its = sum(r["iterations"] for r in runs)
            c1[name] = {"value": its / (sum(r["ms"] for r in runs) / 1e3),
                        "unit": "IPM iters/s", "solves": 2, "warmup_solves": 1,
                        "ms_per_solve": sum(r["ms"] for r in runs) / 2,
                        "iterations_per_solve": its / 2,
                        "objective_error_vs_planted": runs[-1]["objective_error_vs_planted"],
                        "rel_gap": runs[-1]["rel_gap"], "factors": runs[-1]["factors"],
                        "ms_factor_per_solve": runs[-1]["ms_factor"],
                        "ms_solve_per_solve": runs[-1]["ms_solve"],
                        "refine_steps": runs[-1]["refine_steps"]}
            if tuned1:
                c1[name]["autotune"] = tuned1
            q.close()
        c1["mixed_over_fp64"] = c1["mixed"]["value"] / c1["fp64"]["value"]

    # end to end through the C ABI from host memory (headline precision): one
    # step = create from the host LP + one complete solve + x, y, z to pinned
    # host memory + destroy
    e2e = None
    if not args.no_e2e:
        q0 = _blocks(lp)
        n = sum(int(x.n_total) for x in q0)
        m = sum(int(x.m_total) for x in q0)
        xh = torch.empty(n, dtype=torch.float64).pin_memory()
        yh = torch.empty(m, dtype=torch.float64).pin_memory()
        zh = torch.empty(n, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        # the trailing-update kernels the autotuner chose on the headline arm,
        # passed as options the way a caller keeps a tuning result
        kern = {k: int(tuned[k]) for k in ("fp32_update", "ff_update") if k in tuned}
        q = P.arrowhead_lp_create(lp, P.default_options(precision=headline, **opts, **kern))
        _, r = P.ipm_solve(q, out=(xh, yh, zh), check=False)
        if r["status"] != 0:
            raise RuntimeError(f"IPM solve failed: {r}")
        h2d, d2h = P.transfer_bytes(q)
        q.close()
        torch.cuda.synchronize(dev)
        el = max_over_ranks(dist, time.perf_counter() - t0, dev)
        e2e = {"value": replica_value(world, r["iterations"], el * 1e3), "unit": "IPM iters/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "step": f"create from the host LP (upload + symbolic analysis) + one complete "
                       f"solve ({r['iterations']} iterations) + x, y, z to pinned host memory "
                       f"+ destroy, {el:.2f} s; bytes are per solve; trailing-update "
                       f"options {kern or 'default'} (the headline arm's autotuned choice)"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(lp)
    if rank == 0:
        prec = "mixed" if headline == P.PREC_MIXED else "FP64"
        line = {
            "metric": METRIC, "value": value, "unit": "IPM iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if headline == P.PREC_MIXED else "f64", "data": "synthetic",
            "config": {"workload": desc, "parallelism": "replicas" if world > 1 else "single GPU",
                       "step": "one IPM iteration (KKT factor, predictor and corrector solves "
                               "with Krylov refinement, step), timed at iteration boundaries",
                       "l2": "inputs larger than L2 (GBs of block factors per iteration)",
                       "precision": prec, "options": opts},
            "solve": full,
            "clocks": win.clocks, "gpu_launches": win.launches,
            "roofline": roof, "block_factor": factor_roof, "stages": stages,
            "autotune": tuned or None,
            "e2e": e2e, "cpu_baseline": cpu,
            "peaks": peaks,
        }
        line.update({k: v for k, v in summ.items() if k != "ms_per_step"})
        if other_line:
            line["fp64" if other == P.PREC_FP64 else "mixed"] = other_line
            line["mixed_over_fp64"] = (value / other_line["value"] if headline == P.PREC_MIXED
                                       else other_line["value"] / value)
            if full and other_line.get("solve"):
                a, b = full, other_line["solve"]
                mixed, fp = (a, b) if headline == P.PREC_MIXED else (b, a)
                line["mixed_over_fp64_complete_solve"] = fp["ms"] / mixed["ms"]
        if c1:
            line["c1"] = c1
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_kkt(args):
    """KKT factor and solve alone: one factorisation at a seeded interior point
    (x, z = exp(N(0,1)), seed 0) of the first --blocks blocks of the workload,
    then --steps solves (the block solve, Schur solve and back-substitution,
    without Krylov refinement).  Reports the stage times measured with CUDA
    events inside the library."""
    import numpy as np
    import torch
    import paper_2412_07731_gb300 as P
    from instances import prefix
    lp, desc, _ = workload(args.workload)
    if args.blocks and args.blocks < lp.N:
        lp = prefix(lp, args.blocks)
    prec = P.PREC_MIXED if args.precision == "mixed" else P.PREC_FP64
    opts = dict(refine_max=0, fp32_update=args.fp32_update, ff_update=args.ff_update)
    if args.force_fp32:
        opts["fp32_cond_max"] = 1e300
    if args.force_ff:
        opts["fp32_cond_max"] = 1.0
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=prec, **opts))
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(0)
    f64 = dict(dtype=torch.float64, device=dev)
    x = torch.tensor(np.exp(rng.standard_normal(prob.n)), **f64)
    z = torch.tensor(np.exp(rng.standard_normal(prob.n)), **f64)
    rp = torch.tensor(rng.standard_normal(prob.m), **f64)
    zero = torch.zeros(prob.n, **f64)
    fac, sol = [], []
    for _ in range(args.warmup + args.steps):
        P.kkt_factor(prob, x, z)
        fac.append(P.kkt_stage_times(prob))
    for _ in range(args.warmup + args.steps):
        P.kkt_solve(prob, zero, rp, zero)
        sol.append(P.kkt_stage_times(prob)["last_solve_ms"])
    fac, sol = fac[args.warmup:], sol[args.warmup:]
    med = lambda v: statistics.median(v)  # noqa: E731
    line = {"metric": "KKT factor and solve ms", "unit": "ms", "higher_is_better": False,
            "config": {"workload": desc, "blocks": lp.N, "precision": args.precision,
                       "fp32_forced": bool(args.force_fp32), "ff_forced": bool(args.force_ff),
                       "fp32_update": args.fp32_update, "ff_update": args.ff_update,
                       "steps": args.steps,
                       "warmup": args.warmup},
            "form_ms": med([f["form_ms"] for f in fac]),
            "block_factor_ms": med([f["block_factor_ms"] for f in fac]),
            "schur_ms": med([f["schur_ms"] for f in fac]),
            "kkt_solve_ms": med(sol),
            "block_factor_flop": block_factor_flops(lp)}
    print(json.dumps(line), flush=True)
    prob.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c3", "c4", "c1small", "c0"])
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--correctors", type=int, default=0,
                    help="max_correctors of the timed solves (0: plain Mehrotra)")
    ap.add_argument("--other-steps", type=int, default=8,
                    help="timed iterations of the other precision's arm (at most --steps)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the other precision's measurement")
    ap.add_argument("--no-c1", action="store_true", help="skip the 64-block complete solves")
    ap.add_argument("--no-full-solve", action="store_true")
    ap.add_argument("--no-stages", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default trailing-update kernels (no autotuning)")
    ap.add_argument("--kkt-only", action="store_true",
                    help="time one KKT factorisation and --steps solves at a seeded point")
    ap.add_argument("--blocks", type=int, default=0,
                    help="--kkt-only: use the first BLOCKS blocks of the workload")
    ap.add_argument("--force-fp32", action="store_true",
                    help="--kkt-only, mixed: keep FP32 block factors at any conditioning")
    ap.add_argument("--force-ff", action="store_true",
                    help="--kkt-only, mixed: float-float block factors at any conditioning")
    ap.add_argument("--fp32-update", type=int, default=0, choices=[0, 1, 2, 3],
                    help="--kkt-only: trailing update of FP32 factors (0 auto, 1 FP32 pipe, "
                         "2 tensor cores per tile, 3 tensor cores persistent)")
    ap.add_argument("--ff-update", type=int, default=0, choices=[0, 1, 2, 3],
                    help="--kkt-only: trailing update of float-float factors (0 auto, 1 FP32 "
                         "pipe, 2 tensor-core digits per tile, 3 persistent)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.kkt_only:
        run_kkt(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
