"""The multi-rank logic of bench.py on CPU: world_size-2 gloo process groups.

Under torchrun every rank denoises its own image (replicas, weak scaling); the job's
time is the slowest rank's and its throughput counts every rank's units. These tests
run two real ranks over gloo on 127.0.0.1 (no GPU) through the same helpers, and
check that the reference arm's other ranks leave without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_CODE = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import bench
rank, world = dist.get_rank(), dist.get_world_size()
own = [3.5, 7.25][rank]                       # this rank's timed seconds
dist.barrier()
t = bench.max_over_ranks(own, world, "cpu")
rate = bench.job_rate(world, 1000.0, t)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "max": t, "rate": rate}}), flush=True)
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


def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_rate():
    port = _free_port()
    code = RANK_CODE.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        except subprocess.TimeoutExpired:
            p.kill()
            pytest.fail("a gloo rank did not finish")
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["max"] == 7.25                      # the slower rank's time, on every rank
        assert o["rate"] == pytest.approx(2 * 1000.0 / 7.25)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.job_rate(1, 10.0, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    # the oracle arm is a host program: under torchrun the ranks other than 0 exit 0
    # at once without printing (only rank 0 times the oracle and prints its line)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=_env(1, 2, _free_port()), capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
