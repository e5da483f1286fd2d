"""The benchmark's multi-rank host logic on the CPU (gloo, world size 2).

`bench.py --gpus N` under torchrun runs N independent replicas of the
single-GPU path: the ranks meet before the timed region, the job's time is
the slowest rank's (a MAX all-reduce), and the whole-job value counts every
rank's iterations.  The reference arm runs on rank 0 only; other ranks exit
at once without work.
"""
import os
import socket
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RANK_SCRIPT = r"""
import os, sys
sys.path.insert(0, os.getcwd())
import torch.distributed as dist
import bench
rank = int(os.environ["RANK"])
dist.init_process_group("gloo")
dist.barrier()
ms = bench.max_over_ranks(dist, 100.0 + 25.0 * rank)
print("MAX", ms, bench.replica_value(dist.get_world_size(), 20, ms), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return env


def test_slowest_rank_sets_the_job_time():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT], cwd=ROOT,
                              env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.STDOUT, text=True) for r in range(2)]
    outs = []
    try:
        for p in procs:
            out, _ = p.communicate(timeout=180)
            assert p.returncode == 0, out
            outs.append(out)
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    for out in outs:
        line = [x for x in out.splitlines() if x.startswith("MAX")][-1].split()
        assert float(line[1]) == 125.0                     # the slower rank's time
        assert float(line[2]) == 2 * 20 / 0.125            # both ranks' iterations


def test_helpers_without_a_process_group():
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.replica_value(1, 20, 500.0) == 40.0
    assert bench.replica_value(4, 20, 500.0) == 160.0


def test_reference_arm_other_ranks_exit_without_work():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--gpus", "2"], cwd=ROOT, env=_env(1, 2, _free_port()),
                       capture_output=True, text=True, timeout=180)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
