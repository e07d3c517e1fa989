"""Batched denoising of many independent images and the autotuner of its launch.

`Batch` wraps a native batch plan (include/snlm.h, snlm_batch_*): the images'
1-D passes (and the SURE solve/combination) are split into CTA-sized units queued
by dependency level and run by one kernel per class (a pass variant and K, or the
solve and combination), one CTA per unit; the whole run can be captured in a CUDA
graph and replayed.

`autotune` picks the launch parameters of a batch — a cap on CTAs per SM and
the queue order (as given, largest first, smallest first) — by timing graph
replays of the batch itself, and caches the choice per GPU and batch signature.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

from . import api

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "snlm_autotune.json")


def _torch():
    import torch
    return torch


class Batch:
    """One plan over a fixed set of requests. Each request is a dict with keys
    img and out (CUDA tensors), S, K, h (or sigma), and optionally profile,
    order, sigma, beta. Tensors must stay alive and unmoved while the batch is
    used; the workspace is allocated here (PyTorch allocator)."""

    def __init__(self, requests, ctas_per_sm: int = 0, queue_order: int = 0, spin_limit_us: int = 0,
                 fail_job: int = -1, stream=None):
        torch = _torch()
        self.requests = []
        for r in requests:
            r = dict(r)
            if r.get("h") is None:
                r["h"] = api.snlm_default_h(r["sigma"], r["K"], r.get("profile", "box"), r.get("beta", 0.0))
            self.requests.append(r)
        self.stream = stream
        self.plan = api.snlm_batch_plan_create(self.requests, ctas_per_sm, queue_order, spin_limit_us, fail_job)
        dev = self.requests[0]["img"].device
        self.workspace = torch.empty(api.snlm_batch_plan_workspace_bytes(self.plan), dtype=torch.uint8, device=dev)
        api.snlm_batch_plan_upload(self.plan, self.workspace, stream)
        self.captured = False

    def info(self):
        return api.snlm_batch_plan_info(self.plan)

    def run(self, stream=None):
        api.snlm_batch_plan_launch(self.plan, stream if stream is not None else self.stream)

    def capture(self, stream=None):
        """Record one run into a CUDA graph; later runs replay it."""
        torch = _torch()
        st = stream if stream is not None else (self.stream or torch.cuda.current_stream())
        if st == torch.cuda.default_stream():
            st = torch.cuda.Stream()
            st.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(st):
                api.snlm_batch_plan_capture(self.plan, st)
            torch.cuda.current_stream().wait_stream(st)
        else:
            api.snlm_batch_plan_capture(self.plan, st)
        self.captured = True

    def status(self, stream=None) -> int:
        return api.snlm_batch_plan_status(self.plan, stream if stream is not None else self.stream)

    def close(self):
        if self.plan:
            api.snlm_batch_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def signature(requests) -> str:
    """A key for the cache: the multiset of (H, W, dtype, S, K, profile, order)."""
    items = sorted((tuple(r["img"].shape), str(r["img"].dtype), r["S"], r["K"], r.get("profile", "box"),
                    r.get("order", "RC")) for r in requests)
    return hashlib.sha1(repr(items).encode()).hexdigest()[:16]


def time_batch(batch: Batch, reps: int = 5, warmup: int = 2) -> float:
    """Median device time (ms) of one graph-replayed run of the batch."""
    torch = _torch()
    if not batch.captured:
        batch.capture()
    for _ in range(warmup):
        batch.run()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.run()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    if batch.status() != 0:
        raise RuntimeError("batch run reported a timed-out dependency wait")
    return statistics.median(times)


def autotune(requests, candidates=None, reps: int = 5, cache_path: str | None = DEFAULT_CACHE,
             force: bool = False):
    """Choose {ctas_per_sm, queue_order} for this batch by timing graph replays.
    Returns (config, table) where table lists the timings of all candidates."""
    torch = _torch()
    key = f"{torch.cuda.get_device_name()}|{signature(requests)}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache:
        return cache[key]["config"], cache[key]["table"]
    if candidates is None:
        candidates = [dict(ctas_per_sm=c, queue_order=q) for c in (1, 2, 3, 4, 0) for q in (0, 1, 2)]
    table = []
    for cand in candidates:
        b = Batch(requests, **cand)
        try:
            ms = time_batch(b, reps=reps)
        finally:
            b.close()
        table.append(dict(cand, ms=ms))
    best = min(table, key=lambda t: t["ms"])
    config = {k: best[k] for k in ("ctas_per_sm", "queue_order")}
    if cache_path:
        cache[key] = {"config": config, "table": table}
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return config, table
