"""Benchmark: interior-point iterations per second on one GB300.

Workload (default): the uniform-block arrowhead LP with N = 64 blocks, each
A_i 2000 x 3000 with 8 nnz/column (N(0,1) values), 50 linking variables with
5%-dense columns, 20 local link rows per adjacent pair, planted optimum,
seed 1.  One step = one complete interior-point solve to relative gap 1e-8
from Mehrotra's starting point (14 iterations; every iteration runs every
hot-path stage: formation, batched block partial Cholesky with the Schur
contributions, Schur assembly + link-chain/border factor, and the predictor
and corrector solves with their Krylov refinement).  The handle (problem
upload and symbolic analysis) is created before the timed region.

value      IPM iterations/s in mixed precision (FP32 block factors, float-float
           then FP64 ones near the optimum, FP64 Schur complement and
           refinement), inputs resident in device memory
fp64       the same LP and metric with FP64 block factors, beside it
e2e        mixed precision end to end through the C ABI from host memory: each
           step creates the handle from the host LP (upload + symbolic analysis),
           solves, copies x, y, z back and destroys the handle
roofline   the batched block partial Cholesky in the precision that dominates
           the timed solves, against that ALU's peak
cpu_baseline  the CPU oracle (monolithic sparse-LU Mehrotra IPM) timed for one
           IPM iteration on the first block of the same LP, scaled to 64 blocks

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_PEAK_TFLOPS = 1.25       # nominal GB300 FP64 (FMA pipes and DMMA alike)
FP32_PEAK_TFLOPS = 74.7       # GB300 FP32 FMA, measured by the register-only probe
HBM_FALLBACK_GBS = 6800.0     # GB300 copy bandwidth when no measured figure is present


def measured_hbm_gbs() -> float:
    """Copy bandwidth measured on this machine type (MEASURED_PEAKS.json beside
    this file, key hbm_gbs), else the fallback figure."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return HBM_FALLBACK_GBS
METRIC = "IPM iters/s & KKT solve ms at rel. gap 1e-8; mixed vs FP64 GPU path, % peak"


def workload(name: str):
    from instances import config0, config1
    if name == "c1":
        return config1(), "uniform arrowhead LP, N=64 blocks of 2000x3000 (8 nnz/col), " \
                          "n0=50 linking vars (5% dense), l=20 links/pair, planted, FP64"
    if name == "c1small":
        return config1(N=8), "uniform arrowhead LP, N=8 blocks of 2000x3000, n0=50, l=20, FP64"
    if name == "c0":
        return config0(), "tiny arrowhead LP, N=4 blocks of 40x60, n0=3, l=2, FP64"
    raise ValueError(name)


def block_factor_flops(lp) -> float:
    """Algorithmic flops of one batched partial Cholesky: for each block the
    augmented order a = m_i + k_i with m_i pivots; column c costs (a-c-1)
    divides and (a-c-1)(a-c) flops of rank-1 update."""
    N, n0, mg = lp.N, lp.n0, lp.mg
    l = list(int(v) for v in lp.l)
    tot = 0.0
    for i, A in enumerate(lp.A):
        m = A.shape[0]
        k = n0 + mg + (l[i - 1] if i > 0 else 0) + (l[i] if i < N - 1 else 0)
        a = m + k
        # sum_{c=0}^{m-1} (a-c-1) + (a-c-1)(a-c)
        s = 0.0
        for c in range(m):
            r = a - c - 1
            s += r + r * (r + 1)
        tot += s
    return tot


def stage_rooflines(P, prob, lp, hbm_gbs: float):
    """Per-stage times of one KKT factor and one preconditioner application
    (the block solves, the Schur solve and the back-substitution, no Krylov
    refinement) at a seeded interior point (x, z = exp(N(0,1)), seed 0), with
    CUDA events inside the library; median of three after one warm-up.  Each
    stage against the bound that limits it:
      form   -- HBM: the FP32 lower tiles written (pattern reads not counted);
      block  -- FP32 pipe: block_factor_flops against the FP32 FMA probe;
      schur  -- FP64 latency: the link chain is sequential over the link pairs
                and the border is small, so no throughput fraction is claimed;
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
    med = lambda v: statistics.median(v[1:])
    form_ms = med([f["form_ms"] for f in fac])
    block_ms = med([f["block_factor_ms"] for f in fac])
    schur_ms = med([f["schur_ms"] for f in fac])
    apply_ms = med(sol)
    NB = 64
    tiles = 0
    tri = 0
    for i, A in enumerate(lp.A):
        k = lp.n0 + lp.mg + (int(lp.l[i - 1]) if i > 0 else 0) + (int(lp.l[i]) if i < lp.N - 1 else 0)
        a = A.shape[0] + k
        t = (a + NB - 1) // NB
        tiles += t * (t + 1) // 2
        tri += a * (a + 1) // 2
    form_bytes = tiles * NB * NB * 4
    apply_bytes = 2 * tri * 4
    flops = block_factor_flops(lp)
    gbs = lambda b, ms: b / (ms / 1e3) / 1e9
    return {
        "point": "x, z = exp(N(0,1)) (seed 0); FP32 block factors",
        "form": {"ms": form_ms, "bound": "hbm", "bytes": form_bytes,
                 "achieved_gbs": gbs(form_bytes, form_ms),
                 "frac": gbs(form_bytes, form_ms) / hbm_gbs},
        "block_factor": {"ms": block_ms, "bound": "alu (FP32)", "flop": flops,
                         "achieved_tflops": flops / (block_ms / 1e3) / 1e12,
                         "frac": flops / (block_ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS},
        "schur_factor": {"ms": schur_ms, "bound": "FP64 latency (sequential link chain)"},
        "apply": {"ms": apply_ms, "bound": "hbm", "bytes": apply_bytes,
                  "achieved_gbs": gbs(apply_bytes, apply_ms),
                  "frac": gbs(apply_bytes, apply_ms) / hbm_gbs},
        "peaks": {"hbm_gbs": hbm_gbs, "fp32_tflops": FP32_PEAK_TFLOPS},
    }


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


def oracle_iteration_seconds(lp, n_blocks: int = 1):
    """Seconds of one oracle IPM iteration on the first n_blocks of lp."""
    from instances import prefix
    from oracle import ipm, lp as olp
    sub = prefix(lp, n_blocks)
    A, b, c = olp.assemble(sub)
    x, y, z = ipm.starting_point(A, b, c)
    t0 = time.perf_counter()
    ipm.solve(A, b, c, max_iter=1, x0=x, y0=y, z0=z)
    return time.perf_counter() - t0


def cpu_baseline(lp, sample_blocks: int = 1):
    sec = oracle_iteration_seconds(lp, sample_blocks)
    scale = lp.N / sample_blocks
    return {"value": 1.0 / (sec * scale), "unit": "IPM iters/s", "cores": 1, "kind": "oracle",
            "sample": f"one oracle IPM iteration (predictor + corrector, each a SuperLU "
                      f"factorisation of the monolithic augmented system) on the first "
                      f"{sample_blocks} of {lp.N} blocks, {sec:.2f} s, scaled x{scale:g} "
                      f"(linear in blocks; the true growth is superlinear); SuperLU runs on "
                      f"one core"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    lp, desc = workload(args.workload)
    for _ in range(args.warmup):
        oracle_iteration_seconds(lp, 1)
    secs = [oracle_iteration_seconds(lp, 1) for _ in range(args.steps)]
    per_iter = statistics.mean(secs) * lp.N
    value = 1.0 / per_iter
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "IPM iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_iter * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": "IPM iters/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: one oracle IPM iteration on the first of "
                                       f"{lp.N} blocks, scaled x{lp.N}"},
            "e2e": {"value": value, "unit": "IPM iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    lp, desc = workload(args.workload)
    stream = torch.cuda.current_stream(dev)
    headline = P.PREC_MIXED if args.precision == "mixed" else P.PREC_FP64
    other = P.PREC_FP64 if headline == P.PREC_MIXED else P.PREC_MIXED
    # the timed iteration is the plain predictor-corrector step (one factor,
    # predictor and corrector solves); centrality correctors add solves per
    # iteration and do not pay on this well-centred LP (1.16 s vs 1.08 s)
    opts = dict(max_correctors=0)
    prob = P.arrowhead_lp_create(lp, P.default_options(precision=headline, **opts))
    P.load().arrowhead_lp_set_stream(prob.handle, stream.cuda_stream)
    n, m = prob.n, prob.m
    f64 = dict(dtype=torch.float64, device=dev)
    x, y, z = torch.empty(n, **f64), torch.empty(m, **f64), torch.empty(n, **f64)

    def solve():
        _, r = P.ipm_solve(prob, out=(x, y, z), check=False)
        if r["status"] != 0:
            raise RuntimeError(f"IPM solve failed: {r}")
        return r

    def timed(k):
        """k solves between CUDA events on the handle's stream; returns
        (ms, results, launches, clocks)."""
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        sampler = ClockSampler(local)
        l0 = P.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [solve() for _ in range(k)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        launches = P.launch_count() - l0
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        if dist:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
            dist.barrier()
        return ms, res, launches, clocks

    for _ in range(args.warmup):
        solve()
    ms, res, launches, clocks = timed(args.steps)
    iters = sum(r["iterations"] for r in res)
    value = world * iters / (ms / 1e3)

    # roofline: the block partial Cholesky in the precision that took longer
    nf32 = sum(r["factors_fp32"] for r in res)
    nff = sum(r["factors_ff"] for r in res)
    nf64 = sum(r["factors_fp64"] for r in res)
    t32 = sum(r["ms_block_fp32"] for r in res)
    tff = sum(r["ms_block_ff"] for r in res)
    t64 = sum(r["ms_block_fp64"] for r in res)
    flops = block_factor_flops(lp)
    # (count, total ms, peak TFLOP/s, name, peak source) per factor precision;
    # a float-float multiply-add costs about 12 FP32 operations, so its peak
    # in FP64-equivalent flops is the FP32 peak / 12 (the conversion of the
    # FP64 diagonal tiles and panels is not counted in that peak)
    kinds = [(nf32, t32, FP32_PEAK_TFLOPS, "FP32",
              "FP32 FMA register-only probe on this GB300 (profiles/fp64_peak_probe.md)"),
             (nff, tff, FP32_PEAK_TFLOPS / 12.0, "float-float",
              "FP32 FMA probe / 12 FP32 operations per double-float multiply-add"),
             (nf64, t64, FP64_PEAK_TFLOPS, "FP64",
              "nominal GB300 FP64 rate (profiling recipe table); FMA probe measured 1.009 TFLOP/s")]
    cnt, tot, peak, prec_name, peak_src = max(kinds, key=lambda k: k[1] if k[0] else -1.0)
    bf_ms = tot / max(cnt, 1)
    achieved = flops / (bf_ms / 1e3) / 1e12
    other_line = None
    if not args.no_compare:
        P.set_options(prob, P.default_options(precision=other, **opts))
        solve()
        oms, ores, _, oclocks = timed(args.steps)
        oit = sum(r["iterations"] for r in ores)
        other_line = {"precision": "FP64" if other == P.PREC_FP64 else "mixed",
                      "value": world * oit / (oms / 1e3), "unit": "IPM iters/s",
                      "ms_per_step": oms / args.steps, "iterations_per_solve": oit / args.steps,
                      "kkt_factor_ms": sum(r["ms_factor"] for r in ores) / max(oit, 1),
                      "kkt_solve_ms_per_iteration": sum(r["ms_solve"] for r in ores) / max(oit, 1),
                      "refine_steps_per_iteration": sum(r["refine_steps"] for r in ores) / max(oit, 1),
                      "rel_gap": ores[-1]["rel_gap"], "clocks": oclocks}
        P.set_options(prob, P.default_options(precision=headline, **opts))
    stages = None
    if rank == 0 and headline == P.PREC_MIXED:
        stages = stage_rooflines(P, prob, lp, measured_hbm_gbs())
    prob.close()

    # end to end through the C ABI from host memory (mixed precision)
    e2e = None
    if not args.no_e2e:
        xh = torch.empty(n, dtype=torch.float64).pin_memory()
        yh = torch.empty(m, dtype=torch.float64).pin_memory()
        zh = torch.empty(n, dtype=torch.float64).pin_memory()
        h2d = d2h = 0
        eit = 0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            q = P.arrowhead_lp_create(lp, P.default_options(precision=headline, **opts))
            _, r = P.ipm_solve(q, out=(xh, yh, zh), check=False)
            if r["status"] != 0:
                raise RuntimeError(f"IPM solve failed: {r}")
            eit += r["iterations"]
            a, b = P.transfer_bytes(q)
            h2d += a
            d2h += b
            q.close()
        torch.cuda.synchronize(dev)
        el = time.perf_counter() - t0
        if dist:
            t = torch.tensor([el], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": world * eit / el, "unit": "IPM iters/s",
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
               "step": "create from the host LP (upload + symbolic analysis) + solve + "
                       "x, y, z to pinned host memory + destroy"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(lp, 1)
    if rank == 0:
        prec = "mixed" if headline == P.PREC_MIXED else "FP64"
        line = {
            "metric": METRIC, "value": value, "unit": "IPM iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if headline == P.PREC_MIXED else "f64", "data": "synthetic",
            "config": {"workload": desc, "parallelism": "replicas" if world > 1 else "single GPU",
                       "step": "one IPM solve to rel. gap 1e-8 from Mehrotra's starting point",
                       "l2": "inputs larger than L2 (1.1-2.2 GB of block factors per iteration)",
                       "precision": prec, "options": opts},
            "iterations_per_solve": iters / args.steps,
            "rel_gap": res[-1]["rel_gap"],
            "kkt_factor_ms": sum(r["ms_factor"] for r in res) / max(iters, 1),
            "kkt_solve_ms_per_iteration": sum(r["ms_solve"] for r in res) / max(iters, 1),
            "refine_steps_per_iteration": sum(r["refine_steps"] for r in res) / max(iters, 1),
            "factors": {"fp32": nf32 / args.steps, "float_float": nff / args.steps,
                        "fp64": nf64 / args.steps},
            "block_factor_ms": {"fp32": t32 / nf32 if nf32 else None,
                                "float_float": tff / nff if nff else None,
                                "fp64": t64 / nf64 if nf64 else None},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "kernel": f"batched block partial Cholesky ({prec_name}; "
                                   f"pchol_potrf/trsm/update + tinv), {flops:.4g} flop per factor",
                         "peak_source": peak_src},
            "stages": stages,
            "clocks": clocks, "gpu_launches": launches,
            "e2e": e2e, "cpu_baseline": cpu,
        }
        if other_line:
            line["fp64" if other == P.PREC_FP64 else "mixed"] = other_line
            line["mixed_over_fp64"] = (value / other_line["value"] if headline == P.PREC_MIXED
                                       else other_line["value"] / value)
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
    lp, desc = workload(args.workload)
    if args.blocks and args.blocks < lp.N:
        lp = prefix(lp, args.blocks)
    prec = P.PREC_MIXED if args.precision == "mixed" else P.PREC_FP64
    opts = dict(refine_max=0)
    if args.force_fp32:
        opts["fp32_cond_max"] = 1e300
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
    med = lambda v: statistics.median(v)
    line = {"metric": "KKT factor and solve ms", "unit": "ms", "higher_is_better": False,
            "config": {"workload": desc, "blocks": lp.N, "precision": args.precision,
                       "fp32_forced": bool(args.force_fp32), "steps": args.steps,
                       "warmup": args.warmup},
            "form_ms": med([f["form_ms"] for f in fac]),
            "block_factor_ms": med([f["block_factor_ms"] for f in fac]),
            "schur_ms": med([f["schur_ms"] for f in fac]),
            "kkt_solve_ms": med(sol)}
    print(json.dumps(line), flush=True)
    prob.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c1", choices=["c1", "c1small", "c0"])
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the other precision's measurement")
    ap.add_argument("--kkt-only", action="store_true",
                    help="time one KKT factorisation and --steps solves at a seeded point")
    ap.add_argument("--blocks", type=int, default=0,
                    help="--kkt-only: use the first BLOCKS blocks of the workload")
    ap.add_argument("--force-fp32", action="store_true",
                    help="--kkt-only, mixed: keep FP32 block factors at any conditioning")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--probe-peaks", action="store_true",
                    help="build and run the FP64/FP32/TF32 throughput probe, then exit")
    args = ap.parse_args()
    if args.probe_peaks:
        src = os.path.join(ROOT, "paper_2412_07731_gb300", "probe", "peaks.cu")
        exe = os.path.join(ROOT, "paper_2412_07731_gb300", "_build", "peaks_probe")
        os.makedirs(os.path.dirname(exe), exist_ok=True)
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        src], check=True)
        sys.exit(subprocess.run([exe]).returncode)
    if args.kkt_only:
        run_kkt(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
