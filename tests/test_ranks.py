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


SURE_BAND_CODE = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import oracle
from paper_1407_2343_gb300 import shard, synth
rank, world = dist.get_rank(), dist.get_world_size()
sigma, S, K = 20.0, 5, 2
img = synth.noisy_image(61, 44, sigma, seed=3, dtype="f32").astype(np.float64)
h = oracle.default_h(sigma, K)
r0, r1, h0, h1 = shard.band_plan(img.shape[0], world, shard.reach(S, K))[rank]
p = oracle.snlm_parts(img[h0:h1], S, K, h)
sl = slice(r0 - h0, r1 - h0)
f, frc, fcr = img[r0:r1], p["frc"][sl], p["fcr"][sl]
sums = torch.tensor([(frc * frc).sum(), (frc * fcr).sum(), (fcr * fcr).sum(), (f * frc).sum(), (f * fcr).sum(),
                     p["d1"][sl].sum(), p["d2"][sl].sum()], dtype=torch.float64)
dist.all_reduce(sums)                          # the one exchange of a banded SURE run
a11, a12, a22, bf1, bf2, sd1, sd2 = sums.tolist()
b1, b2 = bf1 - sigma ** 2 * sd1, bf2 - sigma ** 2 * sd2
det = a11 * a22 - a12 * a12
theta = [(a22 * b1 - a12 * b2) / det, (a11 * b2 - a12 * b1) / det]
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "theta": theta, "sums": sums.tolist()}}), flush=True)
"""


def test_banded_sure_sums_all_reduce_over_two_gloo_ranks(orc):
    # the exchange step of a single image split into row bands: each rank forms the
    # seven sums of Eqs. (19) and (25) over its own rows (from a crop widened by the
    # passes' reach), one all-reduce adds them, and every rank solves the 2x2 system:
    # the result is the unsharded image's (oracle arithmetic on both sides)
    port = _free_port()
    code = SURE_BAND_CODE.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            p.kill()
            pytest.fail("a gloo rank did not finish")
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    import numpy as np

    from paper_1407_2343_gb300 import synth

    sigma, S, K = 20.0, 5, 2
    img = synth.noisy_image(61, 44, sigma, seed=3, dtype="f32").astype(np.float64)
    _, info = orc.snlm(img, S, K, orc.default_h(sigma, K), order="SURE", sigma=sigma)
    want = [info["A11"], info["A12"], info["A22"], info["sum_f_frc"], info["sum_f_fcr"], info["sum_d1"], info["sum_d2"]]
    for o in outs:
        assert o["sums"] == pytest.approx(want, rel=1e-12)
        assert o["theta"] == pytest.approx([info["theta1"], info["theta2"]], rel=1e-9)


SURE_BAND_GPU_CODE = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
from paper_1407_2343_gb300 import api, shard, synth
rank, world = dist.get_rank(), dist.get_world_size()
dev = torch.device("cuda:0")
sigma, S, K = 25.0, 10, 3
img = torch.from_numpy(synth.noisy_image(333, 270, sigma, seed=4, dtype="u8")).to(dev)
h = api.snlm_default_h(sigma, K)
band = shard.band_plan(img.shape[0], world, shard.reach(S, K))[rank]
f_rc, f_cr, sums = shard.sure_band(img, band, S, K, h)      # the library's own band sums
total = sums.cpu()
dist.all_reduce(total)                                       # the one exchange of a banded SURE run
theta = api.snlm_sure_theta(total.numpy(), sigma)
out = torch.full(img.shape, float("nan"), dtype=torch.float32, device=dev)
shard.sure_finish_band(band, f_rc, f_cr, theta, out)
info = torch.zeros(10, dtype=torch.float64, device=dev)
whole = api.snlm_denoise_ws(img, S, K, h, "box", "SURE", sigma, info=info)
torch.cuda.synchronize()
r0, r1 = band[0], band[1]
err = float((out[r0:r1] - whole[r0:r1]).abs().max())
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "theta": list(theta), "whole_theta": info[:2].tolist(), "err": err}}), flush=True)
"""


@pytest.mark.gpu
def test_banded_sure_with_the_library_sums_over_two_gloo_ranks():
    # two ranks (processes sharing the one GPU, each running its own independent
    # kernels) form the seven sums of their own band with snlm_sure_band; one gloo
    # all-reduce adds them; each solves theta and combines its rows: the result and
    # theta are the unsharded image's
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_2343_gb300 import build

    build.build()
    port = _free_port()
    code = SURE_BAND_GPU_CODE.format(root=ROOT)
    # keep the device selection of this process (CUDA_VISIBLE_DEVICES) for both ranks
    env = [dict(os.environ, RANK=str(r), LOCAL_RANK="0", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                MASTER_PORT=str(port)) for r in range(2)]
    procs = [subprocess.Popen([sys.executable, "-c", code], env=env[r], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            p.kill()
            pytest.fail("a gloo rank did not finish")
        assert p.returncode == 0, e[-3000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["err"] <= 1e-4
        assert o["theta"] == pytest.approx(o["whole_theta"], abs=1e-6)
    assert outs[0]["theta"] == outs[1]["theta"]
