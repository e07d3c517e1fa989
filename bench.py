#!/usr/bin/env python3
"""Benchmark of the separable NLM hot path (Alg. 4 of Ghosh & Chaudhury,
arXiv:1407.2343) on one or more GPUs of one node.

A step is one snlm_denoise of a 4096x4096 uint8 synthetic noisy scene (sigma =
30, S = 20, K = 5, box profile, h = sigma*sqrt(2K+1)) in the SURE order: the four
1-D passes of Alg. 4 with the chained divergence, the 2x2 solve and the
combination. Inputs are resident in HBM when the timed region starts; L2 is
flushed (256 MiB write) between timed steps, outside the per-step events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank denoises its own image
(weak scaling, no data-path collective); value = all ranks' pixels / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "denoised Mpixel/s and lifted patch-pairs/s vs roofline; batched/served vs plain, p50/p99"

# GB300: 152 SMs, 2070 MHz maximum SM clock; per SM per clock: 128 FP32 lanes
# (FADD/FMUL/FFMA each one lane-operation) and 32 MUFU.EX2 results.
SMS, MAX_MHZ = 152, 2070.0
ALU_PEAK_TOPS = SMS * 128 * MAX_MHZ * 1e6 / 1e12
SFU_PEAK_TEXP = SMS * 32 * MAX_MHZ * 1e6 / 1e12
# Algorithmic FP32 operations per unique pair (x, x+s) of one 1-D pass: lift (sub,
# mul) 2, box reduction (add new, remove old) 2, exponent scale 1, accumulation into
# both pixels 4 (two FMA, two adds); the divergence passes add the weighted squared
# differences of both pixels, 2 more. One MUFU ex2 per unique pair.
OPS_PER_PAIR = {"plain": 9, "sure": 11}
# The recursive Gaussian pass (Sec. II-B, Young-van Vliet filter): lift 2, causal
# recursion 4 (B F + three taps), anti-causal recursion 4, exponent scale 1,
# accumulation into both pixels 4; one ex2 per unique pair.
OPS_PER_PAIR_IIR = 15

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# pass kernels of the 4096^2 u8 SURE step, from one ncu capture of those two
# metrics (`-k regex:nlm_pass_kernel -s 12 -c 4`: the first timed step's four
# passes) of `python bench.py --steps 2 --warmup 3 --no-batch --no-serve --no-e2e
# --no-cpu-baseline --no-rc --no-bf --no-nlm2d --no-3d --no-iir --no-fp16
# --no-precision`; valid only while the pass kernels' sources (PASS_KERNEL_SOURCES)
# hash to `sources_sha` (profiles/ has the capture's summary).
TRAFFIC = {"sources_sha": "52540b9a38cf68b2",
           "bytes_per_launch": {"row_pass_sure/slide": 89521152, "col_pass_sure/block": 175208704,
                                "col_pass_sure/slide": 92434176, "row_pass_sure/block": 264592128}}


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks of the process group (a job takes as long as its
    slowest rank); x itself with one rank. `device` holds the reduction tensor: the
    rank's CUDA device under NCCL, the CPU under gloo."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / seconds


# The files the pass kernels are compiled from (their template code, the argument
# and layout structs, and the K = 5 translation unit); the public header supplies
# only status constants to them.
PASS_KERNEL_SOURCES = ("snlm_pass_impl.cuh", "snlm_internal.h", "snlm_pass_k5.cu")


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1407_2343_gb300", "csrc")
    for name in PASS_KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--S", type=int, default=20)
    ap.add_argument("--K", type=int, default=5)
    ap.add_argument("--sigma", type=float, default=30.0)
    ap.add_argument("--dtype", default="u8", choices=["u8", "f16", "f32"])
    ap.add_argument("--order", default="SURE", choices=["RC", "CR", "AVG", "SURE"])
    ap.add_argument("--profile", default="box", choices=["box", "gauss"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-rc", action="store_true", help="skip the extra RC-order measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain measurement")
    ap.add_argument("--no-bf", action="store_true", help="skip the bilateral post-filter measurement")
    ap.add_argument("--no-nlm2d", action="store_true", help="skip the 2-D NLM comparison")
    ap.add_argument("--no-3d", action="store_true", help="skip the separable 3-D extension measurement")
    ap.add_argument("--no-iir", action="store_true", help="skip the recursive Gaussian profile measurement")
    ap.add_argument("--no-fp16", action="store_true", help="skip the fp16-storage measurement")
    ap.add_argument("--no-precision", action="store_true", help="skip the per-configuration error table")
    ap.add_argument("--batch-images", type=int, default=256)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving sweep")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-repeats", type=int, default=3)
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the benchmark line, time Alg. 4 over S (K = 3) and K (S = 20), "
                         "box and Gaussian, and print one JSON line")
    return ap.parse_args()


def workload(a):
    return {"workload": f"{a.size}x{a.size} {a.dtype} synthetic scene (20 shapes + texture + "
                        f"N(0,{a.sigma:g}^2)), S={a.S}, K={a.K}, {a.profile} profile, "
                        f"h=sigma*sqrt(sum g), order {a.order} (Alg. 4)",
            "H": a.size, "W": a.size, "S": a.S, "K": a.K, "sigma": a.sigma, "profile": a.profile,
            "order": a.order, "storage": a.dtype, "seed": 0,
            "l2": "flushed between timed steps (256 MiB write, outside the step events)"}


def passes_of(order):
    return 2 if order in ("RC", "CR") else 4


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"snlm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def cpu_oracle_rate(a, target_s: float, nthreads: int = 0):
    """Time the FP64 oracle (as it stands) on a bounded crop of the workload's
    scene on the host cores (all of them, or `nthreads`); returns (Mpixel/s, cores,
    description, side, seconds)."""
    import oracle
    from paper_1407_2343_gb300 import synth

    oracle.build()
    img = synth.noisy_image(a.size, a.size, a.sigma, seed=0, dtype=a.dtype).astype(np.float64)
    h = oracle.default_h(a.sigma, a.K, a.profile)
    cores = nthreads or oracle.max_threads()
    side = 128 if cores > 1 else 64
    t0 = time.perf_counter()
    oracle.snlm(img[:side, :side], a.S, a.K, h, a.profile, order=a.order, sigma=a.sigma, nthreads=cores)
    t_cal = time.perf_counter() - t0
    side = int(min(a.size, max(64, side * math.sqrt(target_s / max(t_cal, 1e-4)))))
    crop = img[:side, :side]
    t0 = time.perf_counter()
    oracle.snlm(crop, a.S, a.K, h, a.profile, order=a.order, sigma=a.sigma, nthreads=cores)
    dt = time.perf_counter() - t0
    return side * side / dt / 1e6, cores, f"{side}x{side} top-left crop of the same scene, one Alg. 4 run ({dt:.2f} s)", side, dt


def run_reference(a):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1407_2343_gb300 import synth

    oracle.build()
    img = synth.noisy_image(a.size, a.size, a.sigma, seed=0, dtype=a.dtype).astype(np.float64)
    h = oracle.default_h(a.sigma, a.K, a.profile)
    cores = oracle.max_threads()
    # size each step so that the whole run takes about two minutes
    budget = 120.0 / max(1, a.steps + a.warmup)
    side = 96
    t0 = time.perf_counter()
    oracle.snlm(img[:side, :side], a.S, a.K, h, a.profile, order=a.order, sigma=a.sigma)
    t_cal = time.perf_counter() - t0
    side = int(min(a.size, max(64, side * math.sqrt(budget / max(t_cal, 1e-4)))))
    crop = img[:side, :side]
    for _ in range(a.warmup):
        oracle.snlm(crop, a.S, a.K, h, a.profile, order=a.order, sigma=a.sigma)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.snlm(crop, a.S, a.K, h, a.profile, order=a.order, sigma=a.sigma)
    dt = time.perf_counter() - t0
    value = a.steps * side * side / dt / 1e6
    line = {"metric": METRIC, "value": value, "unit": "Mpixel/s", "impl": "reference", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload(a),
            "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                             "sample": f"{side}x{side} top-left crop of the same scene per step"},
            "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_post_filter(a, api, src, flush, stream, step_ms):
    """The bilateral post-filter of Sec. III-B on the step's output (parameters from
    the rules of Sec. IV-A at the scene's sigma): its launch time from the library's
    trace with L2 flushed between launches, its roofline, and SNLM[f] (Alg. 4 then
    the filter) in Mpixel/s."""
    import torch

    ss, sr = api.snlm_bf_params(a.sigma)
    R = int(math.floor(3.0 * float(np.float32(ss))))
    dst = torch.empty_like(src)
    for _ in range(3):
        api.snlm_bilateral(src, ss, sr, out=dst, stream=stream)
    torch.cuda.synchronize()
    n = 50
    api.snlm_trace_read()
    api.snlm_trace_enable(True)
    for _ in range(n):
        flush.zero_()
        api.snlm_bilateral(src, ss, sr, out=dst, stream=stream)
    torch.cuda.synchronize()
    api.snlm_trace_enable(False)
    ms = [m for name, m in api.snlm_trace_read(1 << 16) if name == "bilateral"]
    avg = sum(ms) / len(ms)
    px = src.numel()
    taps = (2 * R + 1) ** 2 - 1
    ops = 5 * taps * px
    achieved = ops / (avg * 1e-3) / 1e12
    return {"sigma_s": ss, "sigma_r": sr, "R": R, "launches": len(ms), "avg_launch_ms": avg,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TOPS,
                         "unit": "Tops/s (FP32 lane-ops)", "frac": achieved / ALU_PEAK_TOPS,
                         "ops_per_tap": 5, "taps_per_pixel": taps,
                         "sfu": {"achieved_Texp_s": taps * px / (avg * 1e-3) / 1e12, "peak_Texp_s": SFU_PEAK_TEXP,
                                 "frac": taps * px / (avg * 1e-3) / 1e12 / SFU_PEAK_TEXP},
                         "dram_bytes_algorithmic": 8 * px},
            "snlm_full_Mpixel_s": px / ((step_ms + avg) * 1e-3) / 1e6}


def measure_nlm2d(a, api, dev, stream, flush):
    """The comparison of the run-time tables of Sec. IV-B on this GPU: the 2-D NLM of
    Eqs. (1)-(2) (S = 20, K = 5, box and Gaussian, evaluated exactly) against Alg. 4
    and SNLM[f] on the same synthetic scenes (N = 256, 512, 1024 and the benchmark's
    size), device times from the library's trace (L2 flushed between launches), and
    the PSNR of each output against the clean scene."""
    import torch
    from paper_1407_2343_gb300 import synth

    S, K, sigma = 20, 5, a.sigma
    rows = []
    for n in sorted({256, 512, 1024, a.size}):
        sc = synth.scene(n, n, sigma, seed=7)
        img = torch.from_numpy(synth.store(sc.noisy, a.dtype)).to(dev)
        out = torch.empty((n, n), dtype=torch.float32, device=dev)
        ws = torch.empty(api.snlm_workspace_bytes(n, n, "SURE"), dtype=torch.uint8, device=dev)
        row = {"N": n}
        for prof in ("box", "gauss"):
            h1 = api.snlm_default_h(sigma, K, prof)
            g = np.exp(-np.arange(-K, K + 1) ** 2 / (2.0 * (K / 2.0) ** 2)) if prof == "gauss" else np.ones(2 * K + 1)
            h2 = sigma * float(g.sum())

            def timed(fn, reps):
                fn()
                torch.cuda.synchronize()
                api.snlm_trace_read()
                api.snlm_trace_enable(True)
                for _ in range(reps):
                    flush.zero_()
                    fn()
                torch.cuda.synchronize()
                api.snlm_trace_enable(False)
                return sum(ms for _, ms in api.snlm_trace_read(1 << 16)) / reps

            reps2 = 2 if n >= 2048 else 5
            t_nlm = timed(lambda: api.snlm_nlm_2d(img, S, K, h2, prof, out=out, stream=stream), reps2)
            psnr_nlm = psnr(out.cpu().numpy(), sc.clean)
            t_snlm = timed(lambda: api.snlm_denoise_ws(img, S, K, h1, prof, "SURE", sigma, out=out, workspace=ws,
                                                       stream=stream), 10)
            psnr_snlm = psnr(out.cpu().numpy(), sc.clean)
            t_full = timed(lambda: api.snlm_denoise_bf(img, S, K, h1, prof, "SURE", sigma, out=out, stream=stream), 10)
            psnr_full = psnr(out.cpu().numpy(), sc.clean)
            row[prof] = {"nlm_2d_ms": t_nlm, "snlm_alg4_ms": t_snlm, "snlm_full_ms": t_full,
                         "speedup_alg4": t_nlm / t_snlm, "speedup_full": t_nlm / t_full,
                         "psnr_noisy": psnr(sc.noisy, sc.clean), "psnr_nlm_2d": psnr_nlm,
                         "psnr_snlm_alg4": psnr_snlm, "psnr_snlm_full": psnr_full}
        rows.append(row)
    return {"S": S, "K": K, "sigma": sigma, "dtype": a.dtype, "rows": rows,
            "note": "2-D NLM evaluated exactly on the GPU (every window offset, separable patch sum); "
                    "h = sigma * sqrt(sum of the patch kernel) for both methods"}


def measure_3d(a, api, dev, stream, flush):
    """The separable 3-D extension on a 256^3 volume (256 frames of the synthetic
    scene at 256^2, the benchmark's storage type, S = 10, K = 3, box): device time
    per call (all its launches, from the library's trace; L2 flushed between calls)
    in the single order XYZ and the average of the six orders."""
    import torch
    from paper_1407_2343_gb300 import synth

    n, S, K = 256, 10, 3
    vol = np.stack([synth.scene(n, n, a.sigma, seed=300 + z).noisy for z in range(n)])
    v = torch.from_numpy(synth.store(vol, a.dtype)).to(dev)
    out = torch.empty((n, n, n), dtype=torch.float32, device=dev)
    h = api.snlm_default_h(a.sigma, K)
    res = {"volume": f"{n}^3 {a.dtype}", "S": S, "K": K}
    for order in ("XYZ", "AVG6"):
        api.snlm_denoise_3d(v, S, K, h, order3=order, out=out, stream=stream)
        torch.cuda.synchronize()
        reps = 5
        api.snlm_trace_read()
        api.snlm_trace_enable(True)
        for _ in range(reps):
            flush.zero_()
            api.snlm_denoise_3d(v, S, K, h, order3=order, out=out, stream=stream)
        torch.cuda.synchronize()
        api.snlm_trace_enable(False)
        tr = api.snlm_trace_read(1 << 16)
        ms = sum(m for _, m in tr) / reps
        res[order] = {"ms": ms, "Mvoxel_s": n ** 3 / (ms * 1e-3) / 1e6, "launches_per_call": len(tr) // reps}
    return res


def measure_iir(a, api, dev, stream, flush):
    """The recursive Gaussian profile (Sec. II-B) against the exact (2K+1)-tap
    Gaussian of Eq. (3) on the benchmark's scene, AVG order (four passes): device
    time per call (from the
    library's launch trace, L2 flushed between calls) at beta = K/2 for K = 2, 5
    and 7, the roofline of the dominant recursive pass, and each output's PSNR
    against the clean scene with their mean difference; then the SURE order of both
    profiles at K = 5 (CUDA events per call)."""
    import torch
    from paper_1407_2343_gb300 import synth

    sc = synth.scene(a.size, a.size, a.sigma, seed=0)
    img = torch.from_numpy(synth.store(sc.noisy, a.dtype)).to(dev)
    clean = torch.from_numpy(sc.clean.astype(np.float32)).to(dev)
    out = torch.empty((a.size, a.size), dtype=torch.float32, device=dev)
    ws = torch.empty(api.snlm_workspace_bytes(a.size, a.size, "AVG"), dtype=torch.uint8, device=dev)
    px = a.size * a.size
    res = {"order": "AVG", "S": a.S, "storage": a.dtype, "cases": []}
    reps = 10
    for K in (2, 5, 7):
        beta = K / 2.0
        case = {"K": K, "beta": beta}
        outs = {}
        for prof in ("gauss_iir", "gauss"):
            h = api.snlm_default_h(a.sigma, K, prof, beta)
            for _ in range(2):
                api.snlm_denoise_ws(img, a.S, K, h, prof, "AVG", 0.0, beta, out=out, workspace=ws, stream=stream)
            torch.cuda.synchronize()
            api.snlm_trace_read()
            api.snlm_trace_enable(True)
            for _ in range(reps):
                flush.zero_()
                api.snlm_denoise_ws(img, a.S, K, h, prof, "AVG", 0.0, beta, out=out, workspace=ws, stream=stream)
            torch.cuda.synchronize()
            api.snlm_trace_enable(False)
            tr = api.snlm_trace_read(1 << 16)
            ms = sum(m for _, m in tr) / reps
            outs[prof] = out.clone()
            c = {"h": h, "ms": ms, "Mpixel_s": px / (ms * 1e-3) / 1e6,
                 "psnr_db": float(10 * math.log10(255.0 ** 2 / float(((out - clean) ** 2).mean())))}
            if prof == "gauss_iir":
                per = {}
                for name, m in tr:
                    per.setdefault(name, []).append(m)
                dom = max(per, key=lambda k: sum(per[k]))
                avg_s = sum(per[dom]) / len(per[dom]) * 1e-3
                pairs = px * a.S
                ach = OPS_PER_PAIR_IIR * pairs / avg_s / 1e12
                c["roofline"] = {"bound": "alu", "kernel": dom, "avg_launch_ms": avg_s * 1e3, "achieved": ach,
                                 "peak": ALU_PEAK_TOPS, "unit": "Tops/s (FP32 lane-ops)", "frac": ach / ALU_PEAK_TOPS,
                                 "ops_per_unique_pair": OPS_PER_PAIR_IIR, "unique_pairs_per_launch": pairs,
                                 "sfu_frac": pairs / avg_s / 1e12 / SFU_PEAK_TEXP}
            case[prof] = c
        case["mean_abs_diff"] = float((outs["gauss_iir"] - outs["gauss"]).abs().mean())
        res["cases"].append(case)
    # the SURE order (all of Alg. 4, with the divergence of Eq. (24)) at K = 5, beta = 2.5
    ws_s = torch.empty(api.snlm_workspace_bytes(a.size, a.size, "SURE"), dtype=torch.uint8, device=dev)
    sure = {"K": 5, "beta": 2.5}
    for prof in ("gauss_iir", "gauss"):
        h = api.snlm_default_h(a.sigma, 5, prof, 2.5)
        for _ in range(2):
            api.snlm_denoise_ws(img, a.S, 5, h, prof, "SURE", a.sigma, 2.5, out=out, workspace=ws_s, stream=stream)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            api.snlm_denoise_ws(img, a.S, 5, h, prof, "SURE", a.sigma, 2.5, out=out, workspace=ws_s, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / reps
        sure[prof] = {"ms": ms, "Mpixel_s": px / (ms * 1e-3) / 1e6,
                      "psnr_db": float(10 * math.log10(255.0 ** 2 / float(((out - clean) ** 2).mean())))}
    res["sure_order"] = sure
    return res


def psnr(x, clean):
    mse = float(np.mean((np.asarray(x, np.float64) - clean) ** 2))
    return 10.0 * math.log10(255.0 ** 2 / mse)


def measure_precision(a, dev):
    """Error of the library against the FP64 oracle, stated per configuration (max-abs
    and mean-abs of the float32 output on the [0, 255] scale; PSNR against the clean
    scene for information):
    - every cell of the 512^2 float32 configuration: sigma in {10, 20, 30, 50} x
      profile {box, Gaussian beta = K/2} x K in {2, 3, 5} x order {RC, CR, AVG,
      SURE}, S = 10, h from the default rule;
    - the large single images in uint8 and float16 storage, 2048^2 and 4096^2, S in
      {10, 20}, K in {3, 5}, box, sigma = 30, SURE order (all four passes), whole
      images."""
    import torch

    import oracle
    from paper_1407_2343_gb300 import api, synth

    oracle.build()
    t0 = time.perf_counter()
    cfg2 = []
    for sigma in (10.0, 20.0, 30.0, 50.0):
        sc = synth.scene(512, 512, sigma, seed=int(sigma))
        f = synth.store(sc.noisy, "f32")
        t = torch.from_numpy(f).to(dev)
        for prof in ("box", "gauss"):
            for K in (2, 3, 5):
                h = api.snlm_default_h(sigma, K, prof, K / 2.0)
                for order in ("RC", "CR", "AVG", "SURE"):
                    got = api.snlm_denoise(t, 10, K, h, prof, order, sigma, K / 2.0).cpu().numpy().astype(np.float64)
                    ref, _ = oracle.snlm(f.astype(np.float64), 10, K, h, prof, K / 2.0, order=order, sigma=sigma)
                    d = np.abs(got - ref)
                    cfg2.append({"sigma": sigma, "profile": prof, "K": K, "order": order,
                                 "max_abs": float(d.max()), "mean_abs": float(d.mean()),
                                 "psnr_db": psnr(got, sc.clean)})
    cfg3 = []
    for n in (2048, 4096):
        sc = synth.scene(n, n, 30.0, seed=0)
        for dt in ("u8", "f16"):
            f = synth.store(sc.noisy, dt)
            t = torch.from_numpy(f).to(dev)
            for S in (10, 20):
                for K in (3, 5):
                    h = api.snlm_default_h(30.0, K)
                    got = api.snlm_denoise(t, S, K, h, "box", "SURE", 30.0).cpu().numpy().astype(np.float64)
                    ref, _ = oracle.snlm(f.astype(np.float64), S, K, h, "box", order="SURE", sigma=30.0)
                    d = np.abs(got - ref)
                    cfg3.append({"size": n, "storage": dt, "S": S, "K": K, "order": "SURE",
                                 "max_abs": float(d.max()), "mean_abs": float(d.mean()),
                                 "psnr_db": psnr(got, sc.clean)})
            del t
    worst = max(c["max_abs"] for c in cfg2 + cfg3)
    return {"tolerance": 1e-4, "worst_max_abs": worst, "cells": len(cfg2) + len(cfg3),
            "config_512_f32": cfg2, "large_u8_f16_sure": cfg3, "seconds": time.perf_counter() - t0}


def measure_storage(a, api, dev, stream, flush, dtype):
    """The benchmark's step (same scene, S, K, order) with the image stored as
    `dtype`: device time per step and the dominant pass's ALU fraction."""
    import torch

    from paper_1407_2343_gb300 import synth

    n = a.size
    img = torch.from_numpy(synth.noisy_image(n, n, a.sigma, seed=0, dtype=dtype)).to(dev)
    out = torch.empty((n, n), dtype=torch.float32, device=dev)
    ws = torch.empty(api.snlm_workspace_bytes(n, n, a.order), dtype=torch.uint8, device=dev)
    h = api.snlm_default_h(a.sigma, a.K, a.profile)

    def step():
        api.snlm_denoise_ws(img, a.S, a.K, h, a.profile, a.order, a.sigma, out=out, workspace=ws, stream=stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    reps = max(10, min(50, a.steps // 8))
    api.snlm_trace_read()
    api.snlm_trace_enable(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in evs:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    api.snlm_trace_enable(False)
    per = {}
    for name, ms in api.snlm_trace_read(1 << 20):
        per.setdefault(name, []).append(ms)
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / reps
    dom = max(per.items(), key=lambda kv: sum(kv[1]))[0]
    avg = float(np.mean(per[dom])) * 1e-3
    kind = "sure" if "_sure" in dom else "plain"
    ach = OPS_PER_PAIR[kind] * n * n * a.S / avg / 1e12
    return {"storage": dtype, "ms_per_step": ms, "Mpixel_s": n * n / (ms * 1e-3) / 1e6,
            "dominant_kernel": dom, "dominant_avg_ms": avg * 1e3, "achieved_Tops": ach,
            "frac_of_nominal": ach / ALU_PEAK_TOPS,
            "kernels_ms": {k: float(np.mean(v)) for k, v in per.items()}}


def measure_batched(a, dev, stream):
    """The uneven batch: images with sides log-uniform in [64, 1024], aspect in
    [1/2, 2], u8/f16, sigma ~ U[10, 50], S in {5,10,15}, K in {2,3,5}, box, RC.
    Plain: one snlm_denoise_ws call per image. Batched: the autotuned persistent
    launch, replayed from a CUDA graph. Both time whole passes over the batch with
    CUDA events; inputs resident, outputs preallocated."""
    import torch

    from paper_1407_2343_gb300 import api, synth
    from paper_1407_2343_gb300.batch import Batch, autotune

    specs = synth.batch_specs(a.batch_images, seed=0)
    reqs = []
    for i, s in enumerate(specs):
        img = torch.from_numpy(synth.noisy_image(s["H"], s["W"], s["sigma"], seed=1000 + i, dtype=s["dtype"])).to(dev)
        reqs.append(dict(img=img, out=torch.empty((s["H"], s["W"]), dtype=torch.float32, device=dev),
                         S=s["S"], K=s["K"], h=api.snlm_default_h(s["sigma"], s["K"]), profile="box",
                         order="RC", sigma=s["sigma"], beta=0.0))
    px = sum(s["H"] * s["W"] for s in specs)
    ws = torch.empty(max(api.snlm_workspace_bytes(s["H"], s["W"], "RC") for s in specs), dtype=torch.uint8, device=dev)
    plain_out = [torch.empty_like(r["out"]) for r in reqs]

    def plain():
        for r, o in zip(reqs, plain_out):
            api.snlm_denoise_ws(r["img"], r["S"], r["K"], r["h"], "box", "RC", r["sigma"], out=o, workspace=ws,
                                stream=stream)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    reps = max(3, min(20, a.steps // 20))
    t_plain = timed(plain, reps)
    cands = [dict(ctas_per_sm=c, queue_order=q) for c in (2, 4, 0) for q in (0, 1)]
    cfg, table = autotune(reqs, candidates=cands, reps=3)
    batch = Batch(reqs, **cfg)
    batch.capture()
    t_batch = timed(batch.run, reps)
    status = batch.status()
    diff = max(float((r["out"] - o).abs().max()) for r, o in zip(reqs, plain_out))
    info = batch.info()
    batch.close()
    n = len(reqs)
    return {"workload": f"{n} uneven images (sides 64..1024 log-uniform, aspect 1/2..2, u8/f16, "
                        f"S in {{5,10,15}}, K in {{2,3,5}}, box, RC), {px / 1e6:.2f} Mpixel in total",
            "plain_images_per_s": n / (t_plain * 1e-3), "batched_images_per_s": n / (t_batch * 1e-3),
            "plain_ms": t_plain, "batched_ms": t_batch, "speedup": t_plain / t_batch,
            "max_abs_diff_batched_vs_plain": diff, "status": status, "config": cfg,
            "autotune_table": table, "plan": info, "reps": reps,
            "plain_gpu_launches_per_pass": 3 * n, "batched_gpu_launches_per_pass": info["classes"]}


def measure_served(a, dev):
    """Poisson arrivals swept from 0.2x to 3x of the plain path's capacity; sizes
    {128, 512, 1024, 2048, 4096}^2 with weights {.3, .3, .2, .15, .05}; each request
    with its own S, K, h, profile and order. The library's serving loop in
    continuous-batching mode against its plain mode (one request at a time through
    the per-image path) on the same schedule; latency is arrival to result in host
    memory. Each point runs `serve_requests` requests `serve_repeats` times (fresh
    schedules, seeds 6, 7, ...); the median and the range over the repeats are
    reported. The timing schedules write their results into a ring of 8 host buffers
    per size (requests of one size share them, so their contents are not checked);
    accuracy is checked on a separate schedule with a buffer per request: served
    against plain (all requests) and against the FP64 oracle (every request up to
    512^2)."""
    import numpy as np
    import torch

    import oracle
    from paper_1407_2343_gb300 import api, serve

    n, reps = a.serve_requests, a.serve_repeats
    pool = serve.make_pool()
    ring = {sz: [torch.empty((sz, sz), dtype=torch.float32).pin_memory() for _ in range(8)] for sz in serve.SIZES}

    def schedule(rate, seed, count=n):
        sched = serve.make_schedule(count, rate=rate, seed=seed, pool=pool)
        used = {}
        for r in sched:
            k = used.get(r.shape[0], 0)
            r.out = ring[r.shape[0]][k % 8]
            used[r.shape[0]] = k + 1
        return sched

    plain_srv, served_srv = serve.NativeServer("plain"), serve.NativeServer("batched")
    # warm-up of both loops: every kernel variant a schedule can reach is loaded and
    # configured once (each combination of S, K, profile, order and storage, on the
    # batched path at 128^2 and on the per-image path at 1024^2), then a random mix
    warm = []
    for sz in (128, 1024):
        for S in (5, 10, 15, 20):
            for K in (2, 3, 5):
                for prof in ("box", "gauss"):
                    for order in ("RC", "CR", "AVG", "SURE"):
                        for k in (0, 1):
                            img, sigma = pool[(sz, k)]
                            h = api.snlm_default_h(sigma, K, prof, K / 2.0)
                            warm.append(serve.Request(len(warm), img, S, K, h, prof, order, sigma, K / 2.0, 0.0))
    for srv in (plain_srv, served_srv):
        srv.run(serve.prepare_outputs(warm))
        srv.run(schedule(1e9, 4, min(n, 400)))
    # capacity of the plain path: everything arrives at once (best of two runs)
    cap = 0.0
    for k in range(2):
        cap = max(cap, plain_srv.run(schedule(1e9, 5 + k)).summary()["images_per_s"])
    sweep = []
    for frac in (0.2, 0.5, 1.0, 1.5, 2.0, 3.0):
        rate = frac * cap
        runs = {"plain": [], "served": []}
        for rep in range(reps):
            for mode, srv in (("plain", plain_srv), ("served", served_srv)):
                runs[mode].append(srv.run(schedule(rate, 6 + rep)).summary())
        pt = {"rate_frac_of_plain_capacity": frac, "rate_per_s": rate}
        for mode in ("plain", "served"):
            agg = {}
            for key in ("images_per_s", "p50_ms", "p99_ms", "mean_ms"):
                v = [r[key] for r in runs[mode]]
                agg[key] = float(np.median(v))
                agg[key + "_range"] = [float(min(v)), float(max(v))]
            sizes = sorted({k for r in runs[mode] for k in r["by_size"]}, key=int)
            agg["p99_ms_by_size"] = {k: float(np.median([r["by_size"][k]["p99_ms"] for r in runs[mode]
                                                         if k in r["by_size"]])) for k in sizes}
            agg["loop_max_yield_ms"] = max(r["loop"].get("max_yield_ms", 0.0) for r in runs[mode])
            agg["loop_max_iter_ms"] = max(r["loop"].get("max_iter_ms", 0.0) for r in runs[mode])
            agg["loop_yields_over_1ms"] = sum(r["loop"].get("yields_over_1ms", 0) for r in runs[mode])
            agg["max_batch"] = max(r["max_batch"] for r in runs[mode])
            agg["max_inflight_steps"] = max(r["max_inflight_steps"] for r in runs[mode])
            pt[mode] = agg
        sweep.append(pt)
    # accuracy: a separate schedule at 2x capacity, one result buffer per request
    n_acc = 120
    sp = serve.prepare_outputs(serve.make_schedule(n_acc, rate=2 * cap, seed=99, pool=pool))
    ss = serve.prepare_outputs(serve.make_schedule(n_acc, rate=2 * cap, seed=99, pool=pool))
    plain_srv.run(sp)
    served_srv.run(ss)
    worst_vs_plain = max(float(np.abs(x.out.numpy() - y.out.numpy()).max()) for x, y in zip(sp, ss))
    worst_vs_oracle, checked = 0.0, 0
    for r in ss:
        if r.shape[0] > 512:
            continue
        ref, _ = oracle.snlm(r.img.numpy().astype(np.float64), r.S, r.K, r.h, r.profile, r.beta, r.order, r.sigma)
        worst_vs_oracle = max(worst_vs_oracle, float(np.abs(r.out.numpy() - ref).max()))
        checked += 1
    return {"workload": f"{n} requests per point, {reps} repeats (median and range), Poisson arrivals, sizes "
                        "128..4096 squared with weights .3/.3/.2/.15/.05, S in {5,10,15,20}, K in {2,3,5}, "
                        "box/gauss, RC/CR/AVG/SURE, u8/f16",
            "plain_capacity_images_per_s": cap, "sweep": sweep,
            "accuracy_schedule_requests": n_acc, "max_abs_served_vs_plain": worst_vs_plain,
            "max_abs_served_vs_oracle": worst_vs_oracle, "oracle_checked_requests": checked}


def run_ours(a):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_1407_2343_gb300 import _lib, api, synth

    _lib.load(build_if_missing=True)
    img_np = synth.noisy_image(a.size, a.size, a.sigma, seed=rank, dtype=a.dtype)
    img = torch.from_numpy(img_np).to(dev)
    H = W = a.size
    h = api.snlm_default_h(a.sigma, a.K, a.profile)
    out = torch.empty((H, W), dtype=torch.float32, device=dev)
    ws = torch.empty(api.snlm_workspace_bytes(H, W, a.order), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(order=a.order):
        api.snlm_denoise_ws(img, a.S, a.K, h, a.profile, order, a.sigma, out=out, workspace=ws, stream=stream)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    # measured FP32 and MUFU.EX2 rates of this GPU (the library's probe kernels),
    # taken before the timed region
    peaks = api.snlm_probe_peaks(stream)
    fp32_meas = max(peaks["fp32_fma2_ops_s"], peaks["fp32_fma_ops_s"]) / 1e12
    ex2_meas = peaks["ex2_s"] / 1e12

    def timed(order, steps, clocks=None):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        api.snlm_trace_read()
        api.snlm_trace_enable(True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        w0 = time.perf_counter()
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(stream)
            step(order)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - w0
        ck = clocks.stop() if clocks else None
        api.snlm_trace_enable(False)
        trace = api.snlm_trace_read(1 << 20)
        dev_ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        return dev_ms, wall, trace, ck

    dev_ms, wall, trace, clocks = timed(a.order, a.steps, Clocks(local))
    dev_ms_max = max_over_ranks(dev_ms, world, dev)
    px = H * W
    value = job_rate(world, a.steps * px, dev_ms_max * 1e-3) / 1e6
    npass = passes_of(a.order)
    pairs_paper = world * a.steps * npass * px * (2 * a.S + 1) / (dev_ms_max * 1e-3)

    # per-kernel times from the launch trace (CUDA events on the launching stream)
    per = {}
    for name, ms in trace:
        d = per.setdefault(name, [0, 0.0])
        d[0] += 1
        d[1] += ms
    total_k = sum(v[1] for v in per.values()) or 1.0
    kernels = {k: {"launches": v[0], "total_ms": v[1], "avg_ms": v[1] / v[0], "share": v[1] / total_k}
               for k, v in sorted(per.items(), key=lambda kv: -kv[1][1])}
    dom = max(per.items(), key=lambda kv: kv[1][1])[0]
    avg_s = per[dom][1] / per[dom][0] * 1e-3
    kind = "sure" if "_sure" in dom else "plain"
    pairs_launch = px * a.S
    achieved = OPS_PER_PAIR[kind] * pairs_launch / avg_s / 1e12
    traffic = None
    if TRAFFIC["sources_sha"] == kernel_sources_sha() and a.size == 4096 and a.S == 20 and a.K == 5 and \
            a.dtype == "u8" and a.profile == "box":
        traffic = TRAFFIC["bytes_per_launch"].get(dom)
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": ALU_PEAK_TOPS,
                "unit": "Tops/s (FP32 lane-ops)", "frac": achieved / ALU_PEAK_TOPS, "traffic": traffic,
                "ops_per_unique_pair": OPS_PER_PAIR[kind], "unique_pairs_per_launch": pairs_launch,
                "avg_launch_ms": avg_s * 1e3,
                "sfu": {"achieved_Texp_s": pairs_launch / avg_s / 1e12, "peak_Texp_s": SFU_PEAK_TEXP,
                        "frac": pairs_launch / avg_s / 1e12 / SFU_PEAK_TEXP,
                        "measured_peak_Texp_s": ex2_meas, "frac_of_measured": pairs_launch / avg_s / 1e12 / ex2_meas},
                "peak_source": "152 SMs x 128 FP32 lanes x 2070 MHz (unit counts and maximum clock)",
                "measured_peak": fp32_meas, "frac_of_measured": achieved / fp32_meas,
                "measured_peak_source": "snlm_probe_peaks: independent FMA chains in every thread of 8 CTAs x 256 "
                                        "threads per SM (best of packed FP32x2 and scalar FMA), CUDA events",
                "probe": {k: v / 1e12 for k, v in peaks.items()}}

    line = {"metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": dev_ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload(a), "parallelism": f"replicas{world}" if world > 1 else "single",
            "pairs_per_s": pairs_paper, "unique_pairs_per_s": pairs_paper * a.S / (2 * a.S + 1),
            "wall_s_timed_region": wall, "roofline": roofline, "kernels": kernels,
            "gpu_launches": len(trace), "clocks": clocks}

    if not a.no_rc and a.order != "RC":
        n_rc = max(20, a.steps // 4)
        ms_rc, _, tr_rc, _ = timed("RC", n_rc)
        ms_rc = max_over_ranks(ms_rc, world, dev)
        line["rc_order"] = {"Mpixel_s": job_rate(world, n_rc * px, ms_rc * 1e-3) / 1e6, "ms_per_step": ms_rc / n_rc,
                            "gpu_launches": len(tr_rc)}

    if not a.no_e2e:
        # end to end through the pipelined host-buffer entry point: every step copies
        # its own input in from pinned host memory and its result out into its own
        # pinned buffer; the copies overlap the neighbouring steps' computation. Two
        # different scenes alternate (the first is the device-timed one).
        n_e2e = max(24, a.steps // 10)
        img2 = synth.noisy_image(a.size, a.size, a.sigma, seed=rank + 1000, dtype=a.dtype)
        host_in = [torch.from_numpy(img_np).pin_memory(), torch.from_numpy(img2).pin_memory()]
        ring = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(8)]
        ins = [host_in[k % 2] for k in range(n_e2e)]
        outs = [ring[k % 8] for k in range(n_e2e)]
        step()
        torch.cuda.synchronize()
        dev_ref = out.cpu()
        api.snlm_denoise_host_many(ins[:2], a.S, a.K, h, a.profile, a.order, a.sigma, outs=outs[:2], stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.snlm_denoise_host_many(ins, a.S, a.K, h, a.profile, a.order, a.sigma, outs=outs, stream=stream)
        t_many = max_over_ranks(time.perf_counter() - t0, world, dev)
        same = bool(torch.equal(outs[n_e2e - 2], dev_ref))      # an even step: the device-timed scene
        # one synchronous host-to-host call per step, for comparison
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            api.snlm_denoise_host(ins[k], a.S, a.K, h, a.profile, a.order, a.sigma, out=outs[k], stream=stream)
        t_single = max_over_ranks(time.perf_counter() - t0, world, dev)
        line["e2e"] = {"value": job_rate(world, n_e2e * px, t_many) / 1e6, "unit": "Mpixel/s",
                       "h2d_bytes_per_step": int(img_np.nbytes), "d2h_bytes_per_step": int(H * W * 4),
                       "steps": n_e2e, "api": "snlm_denoise_host_many (pinned host buffers, copies overlapped "
                                              "with the neighbouring steps' computation)",
                       "result_equals_device_path": same,
                       "single_call": {"value": job_rate(world, n_e2e * px, t_single) / 1e6, "unit": "Mpixel/s",
                                       "api": "snlm_denoise_host, one synchronous call per step"}}

    if not a.no_bf:
        step()
        line["post_filter"] = measure_post_filter(a, api, out, flush, stream, dev_ms_max / a.steps)

    if not a.no_nlm2d and rank == 0:
        line["nlm_2d_comparison"] = measure_nlm2d(a, api, dev, stream, flush)

    if not a.no_3d and rank == 0:
        line["volume_3d"] = measure_3d(a, api, dev, stream, flush)

    if not a.no_iir and rank == 0:
        line["gauss_iir"] = measure_iir(a, api, dev, stream, flush)

    if not a.no_batch:
        line["batched"] = measure_batched(a, dev, stream)

    if not a.no_serve and rank == 0:
        line["served"] = measure_served(a, dev)

    if not a.no_fp16 and rank == 0:
        line["fp16_storage"] = measure_storage(a, api, dev, stream, flush, "f16")

    if not a.no_precision and rank == 0:
        line["precision"] = measure_precision(a, dev)

    if rank == 0 and not a.no_cpu_baseline:
        v, cores, desc, _, _ = cpu_oracle_rate(a, target_s=6.0)
        v1, _, desc1, _, _ = cpu_oracle_rate(a, target_s=4.0, nthreads=1)
        line["cpu_baseline"] = {"value": v, "unit": "Mpixel/s", "cores": cores, "kind": "oracle", "sample": desc,
                                "single_core": {"value": v1, "unit": "Mpixel/s", "cores": 1, "sample": desc1}}

    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(summary_line(line), flush=True)
        print(json.dumps(line), flush=True)


def summary_line(line):
    """One human-readable line of the headline figures (printed just before the JSON)."""
    parts = [f"summary: {line['value']:.0f} Mpixel/s ({line['ms_per_step']:.3f} ms/step)",
             f"dominant {line['roofline']['kernel']} {line['roofline']['avg_launch_ms']:.3f} ms = "
             f"{line['roofline']['frac']:.3f} of nominal ALU, {line['roofline']['frac_of_measured']:.3f} of measured"]
    if "e2e" in line:
        parts.append(f"e2e {line['e2e']['value']:.0f} Mpixel/s")
    if "fp16_storage" in line:
        parts.append(f"fp16 {line['fp16_storage']['Mpixel_s']:.0f} Mpixel/s")
    if "batched" in line:
        b = line["batched"]
        parts.append(f"batched {b['batched_images_per_s']:.0f} vs plain {b['plain_images_per_s']:.0f} images/s "
                     f"({b['speedup']:.2f}x)")
    if "served" in line:
        pts = []
        for p in line["served"]["sweep"]:
            pts.append(f"{p['rate_frac_of_plain_capacity']:g}x: {p['served']['images_per_s']:.0f}/"
                       f"{p['plain']['images_per_s']:.0f} img/s p99 {p['served']['p99_ms']:.2f}/"
                       f"{p['plain']['p99_ms']:.2f} ms")
        parts.append("served/plain " + "; ".join(pts))
    if "precision" in line:
        parts.append(f"worst max-abs vs oracle {line['precision']['worst_max_abs']:.2e} over "
                     f"{line['precision']['cells']} cells")
    if "cpu_baseline" in line:
        parts.append(f"oracle {line['cpu_baseline']['value']:.2f} Mpixel/s on {line['cpu_baseline']['cores']} cores, "
                     f"{line['cpu_baseline']['single_core']['value']:.3f} on 1")
    return " | ".join(parts)


def run_sweep(a):
    """Run time of Alg. 4 (the SURE order, all four passes) against the search and
    patch half-widths, the scaling study of the run-time figure of Sec. IV-B: S in
    {10, 15, 20, 25, 30} at K = 3 and K in {2, ..., 7} at S = 20, box and Gaussian,
    on the benchmark's scene; device time per step from CUDA events (L2 flushed
    between steps), median of the steps."""
    import torch
    from paper_1407_2343_gb300 import _lib, api, synth

    _lib.load(build_if_missing=True)
    dev = torch.device("cuda", 0)
    n = a.size
    img = torch.from_numpy(synth.noisy_image(n, n, a.sigma, seed=0, dtype=a.dtype)).to(dev)
    out = torch.empty((n, n), dtype=torch.float32, device=dev)
    ws = torch.empty(api.snlm_workspace_bytes(n, n, a.order), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    points = [(S, 3) for S in (10, 15, 20, 25, 30)] + [(20, K) for K in (2, 3, 4, 5, 6, 7)]
    rows = []
    for prof in ("box", "gauss"):
        for S, K in points:
            h = api.snlm_default_h(a.sigma, K, prof)

            def step():
                api.snlm_denoise_ws(img, S, K, h, prof, a.order, a.sigma, out=out, workspace=ws, stream=stream)

            for _ in range(3):
                step()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
            for e0, e1 in evs:
                flush.zero_()
                e0.record(stream)
                step()
                e1.record(stream)
            torch.cuda.synchronize()
            ms = float(np.median([e0.elapsed_time(e1) for e0, e1 in evs]))
            rows.append({"profile": prof, "S": S, "K": K, "ms": ms, "Mpixel_s": n * n / (ms * 1e-3) / 1e6})
    print(json.dumps({"sweep": "Alg. 4 run time against S and K", "size": n, "dtype": a.dtype, "order": a.order,
                      "rows": rows}), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.sweep:
        run_sweep(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
