"""Continuous-batching service for denoise requests, and its plain per-request
counterpart.

A request carries its own image (host memory), S, K, h, profile and order. The
server replays an arrival schedule against the wall clock and loops:

1. admission: arrived requests are admitted in arrival order while their device
   footprint (input, output, their scratch) fits the memory budget (a fraction of
   the free HBM when the server starts, or an explicit cap); the input is copied
   host-to-device on an upload stream;
2. launch: admitted requests of at least `solo_pixels` pixels run alone through the
   per-image path (they fill the GPU by themselves), each on its own stream with its
   own workspace; the smaller ones become one batch plan (the native persistent
   launch over their tile units) — or run alone too when one small request finds
   the GPU idle, which keeps the latency of a quiet server at the per-image path's.
   Up to `streams` launches are in flight, so work that arrives meanwhile overlaps
   with them on the GPU;
3. retirement: every finished launch (in completion order) has its outputs copied
   back to pinned host buffers, its memory released and each request's latency
   (arrival to result in host memory) recorded.

The plain path serves the same schedule one request at a time with
snlm_denoise_host-style calls (copy in, denoise, copy out).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import api, synth

SIZES = (128, 512, 1024, 2048, 4096)
SIZE_WEIGHTS = (0.3, 0.3, 0.2, 0.15, 0.05)


@dataclass
class Request:
    rid: int
    img: object                 # pinned host tensor (H, W): uint8 / float16 / float32
    S: int
    K: int
    h: float
    profile: str
    order: str
    sigma: float
    beta: float
    t_arrival: float            # seconds from the start of the schedule
    # filled by a run (preallocated by prepare_outputs, outside any timed region)
    out: object = None          # pinned host float32 result
    t_done: float = math.nan
    step: int = -1

    @property
    def shape(self):
        return tuple(self.img.shape)

    def latency(self):
        return self.t_done - self.t_arrival


def make_pool(sizes=SIZES, pool_per_size: int = 2, pin: bool = True):
    """A small pool of synthetic noisy scenes per size (u8 and f16), shared by
    the requests of a schedule (read-only)."""
    import torch

    pool = {}
    for s in sizes:
        for k in range(pool_per_size):
            sigma = 10.0 + 40.0 * ((k + 1) / (pool_per_size + 1))
            dt = "u8" if k % 2 == 0 else "f16"
            img = torch.from_numpy(synth.noisy_image(s, s, sigma, seed=10 * s + k, dtype=dt))
            pool[(s, k)] = (img.pin_memory() if pin else img, sigma)
    return pool


def make_schedule(n: int, rate: float, seed: int = 0, sizes=SIZES, weights=SIZE_WEIGHTS, pool_per_size: int = 2,
                  pin: bool = True, pool=None):
    """n requests with Poisson arrivals at `rate` per second. Images come from a
    small pool of synthetic scenes per size (shared, read-only); each request
    draws its own S, K, profile, order and sigma (h from the default rule)."""
    rng = np.random.default_rng(seed)
    if pool is None:
        pool = make_pool(sizes, pool_per_size, pin)
    t = 0.0
    reqs = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        s = int(rng.choice(sizes, p=np.asarray(weights) / np.sum(weights)))
        img, sigma = pool[(s, int(rng.integers(pool_per_size)))]
        S = int(rng.choice([5, 10, 15, 20]))
        K = int(rng.choice([2, 3, 5]))
        profile = str(rng.choice(["box", "gauss"]))
        order = str(rng.choice(["RC", "CR", "AVG", "SURE"]))
        beta = K / 2.0
        h = api.snlm_default_h(sigma, K, profile, beta)   # the library's default rule
        reqs.append(Request(i, img, S, K, h, profile, order, sigma, beta, t))
    return reqs


def prepare_outputs(schedule, pin: bool = True):
    """Allocate every request's host result buffer (pinned) ahead of a run."""
    import torch

    for r in schedule:
        if r.out is None or tuple(r.out.shape) != r.shape:
            o = torch.empty(r.shape, dtype=torch.float32)
            r.out = o.pin_memory() if pin else o
    return schedule


def _footprint(r: Request) -> int:
    H, W = r.shape
    # input + output + the batch scratch of the request (intermediates of its order)
    return r.img.element_size() * H * W + 4 * H * W + api.snlm_workspace_bytes(H, W, r.order)


@dataclass
class ServeStats:
    latencies: list = field(default_factory=list)
    sizes: list = field(default_factory=list)      # image height of each latency
    steps: int = 0
    max_inflight: int = 0
    max_batch: int = 0
    wall: float = 0.0
    images: int = 0
    max_used: int = 0           # peak device bytes of admitted requests
    host_s: dict = field(default_factory=lambda: {"admit": 0.0, "launch": 0.0, "retire": 0.0})
    loop: dict = field(default_factory=dict)        # native loop: longest yield and work pass

    def summary(self):
        lat = np.asarray(self.latencies) * 1e3
        return {"images": self.images, "wall_s": self.wall, "images_per_s": self.images / self.wall if self.wall else 0,
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "mean_ms": float(lat.mean()) if len(lat) else None, "steps": self.steps,
                "max_batch": self.max_batch, "max_inflight_steps": self.max_inflight,
                "peak_admitted_bytes": self.max_used,
                "host_ms": {k: v * 1e3 for k, v in self.host_s.items()},
                "by_size": self.by_size(), "loop": dict(self.loop)}

    def by_size(self):
        """Count, p50 and p99 of the latencies (ms) per image height."""
        lat = np.asarray(self.latencies) * 1e3
        sz = np.asarray(self.sizes)
        out = {}
        if len(sz) != len(lat):
            return out
        for v in sorted(set(self.sizes)):
            x = lat[sz == v]
            out[str(v)] = {"n": int(len(x)), "p50_ms": float(np.percentile(x, 50)),
                           "p99_ms": float(np.percentile(x, 99))}
        return out


class Server:
    """The continuous-batching loop (single host thread)."""

    def __init__(self, device=None, mem_budget: int | None = None, mem_fraction: float = 0.5, streams: int = 4,
                 max_batch: int = 256, ctas_per_sm: int = 0, solo_pixels: int = 1024 * 1024):
        import torch

        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        free, _ = torch.cuda.mem_get_info(self.dev)
        self.budget = int(mem_budget if mem_budget is not None else free * mem_fraction)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(max(1, streams))]
        self.upload = torch.cuda.Stream(self.dev)
        self.max_batch = max_batch
        self.ctas_per_sm = ctas_per_sm
        self.solo_pixels = solo_pixels

    def _launch_solo(self, item, st):
        import torch

        r, d_in, d_out, ev, _ = item
        st.wait_event(ev)
        with torch.cuda.stream(st):
            ws = torch.empty(api.snlm_workspace_bytes(r.shape[0], r.shape[1], r.order), dtype=torch.uint8,
                             device=self.dev)
            api.snlm_denoise_ws(d_in, r.S, r.K, r.h, r.profile, r.order, r.sigma, r.beta, out=d_out, workspace=ws,
                                stream=st)
            done = torch.cuda.Event()
            done.record(st)
        return {"batch": None, "keep": ws, "done": done, "members": [item], "stream": st}

    def _launch_batch(self, items, st):
        import torch

        from .batch import Batch

        for (_, _, _, ev, _) in items:
            st.wait_event(ev)
        reqs = [dict(img=d_in, out=d_out, S=r.S, K=r.K, h=r.h, profile=r.profile, order=r.order,
                     sigma=r.sigma, beta=r.beta) for (r, d_in, d_out, _, _) in items]
        with torch.cuda.stream(st):
            b = Batch(reqs, ctas_per_sm=self.ctas_per_sm, stream=st)
            b.run(st)
            # the run's failure word lands in pinned memory behind it: read after `done`
            word = torch.zeros(1, dtype=torch.int32).pin_memory()
            api.snlm_batch_plan_status_async(b.plan, word, st)
            done = torch.cuda.Event()
            done.record(st)
        return {"batch": b, "keep": None, "done": done, "members": items, "stream": st, "word": word}

    def run(self, schedule, stats: ServeStats | None = None):
        import torch

        stats = stats or ServeStats()
        prepare_outputs(schedule)
        pending = list(schedule)          # in arrival order
        pi = 0
        admitted = []                     # (req, dev_in, dev_out, upload event, bytes)
        inflight = []                     # launches: dicts of _launch_solo / _launch_batch
        used = 0
        t0 = time.perf_counter()
        while pi < len(pending) or admitted or inflight:
            now = time.perf_counter() - t0
            h0 = time.perf_counter()
            # 1. admission
            while pi < len(pending) and pending[pi].t_arrival <= now and len(admitted) < self.max_batch:
                r = pending[pi]
                need = _footprint(r)
                if need > self.budget:
                    raise ValueError(f"request {r.rid} needs {need} bytes, more than the whole budget")
                if used + need > self.budget:
                    break                 # wait for memory to free up
                with torch.cuda.stream(self.upload):
                    d_in = r.img.to(self.dev, non_blocking=True)
                    d_out = torch.empty(r.shape, dtype=torch.float32, device=self.dev)
                    ev = torch.cuda.Event()
                    ev.record(self.upload)
                used += need
                stats.max_used = max(stats.max_used, used)
                admitted.append((r, d_in, d_out, ev, need))
                pi += 1
            h1 = time.perf_counter()
            stats.host_s["admit"] += h1 - h0
            # 2. launches on the free streams: large requests alone, the rest batched
            if admitted:
                busy = {id(e["stream"]) for e in inflight}
                free_streams = [st for st in self.streams if id(st) not in busy]
                large = [a for a in admitted if a[0].shape[0] * a[0].shape[1] >= self.solo_pixels]
                small = [a for a in admitted if a[0].shape[0] * a[0].shape[1] < self.solo_pixels]
                if len(small) == 1 and not inflight and not large:
                    large, small = small, []          # a lone request on an idle GPU
                launched = []

                def start(e):
                    for (r, _, _, _, _) in e["members"]:
                        r.step = stats.steps
                    stats.steps += 1
                    stats.max_batch = max(stats.max_batch, len(e["members"]))
                    inflight.append(e)
                    launched.extend(e["members"])

                for a in large:
                    if not free_streams:
                        break
                    start(self._launch_solo(a, free_streams.pop(0)))
                if small and free_streams:
                    start(self._launch_batch(small, free_streams.pop(0)))
                if launched:
                    ids = {id(a) for a in launched}
                    admitted = [a for a in admitted if id(a) not in ids]
                stats.max_inflight = max(stats.max_inflight, len(inflight))
            h2 = time.perf_counter()
            stats.host_s["launch"] += h2 - h1
            # 3. retire every finished launch
            keep = []
            for e in inflight:
                if not e["done"].query():
                    keep.append(e)
                    continue
                st = e["stream"]
                if e["batch"] is not None and int(e["word"][0]) != 0:
                    raise RuntimeError("a batch step reported a timed-out dependency wait")
                with torch.cuda.stream(st):
                    for (r, d_in, d_out, _, need) in e["members"]:
                        r.out.copy_(d_out, non_blocking=True)
                st.synchronize()
                t_done = time.perf_counter() - t0
                for (r, d_in, d_out, _, need) in e["members"]:
                    r.t_done = t_done
                    stats.latencies.append(r.latency())
                    stats.sizes.append(r.shape[0])
                    used -= need
                stats.images += len(e["members"])
                if e["batch"] is not None:
                    e["batch"].close()
            inflight = keep
            stats.host_s["retire"] += time.perf_counter() - h2
            if pi < len(pending) and not admitted and not inflight:
                # idle until the next arrival
                wait = pending[pi].t_arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.002))
        stats.wall = time.perf_counter() - t0
        return stats


def run_plain(schedule, device=None, stats: ServeStats | None = None):
    """Serve the schedule one request at a time (FIFO): copy in, snlm_denoise,
    copy out, wait."""
    import torch

    dev = device or torch.device("cuda", torch.cuda.current_device())
    stats = stats or ServeStats()
    prepare_outputs(schedule)
    st = torch.cuda.Stream(dev)
    t0 = time.perf_counter()
    for r in schedule:
        now = time.perf_counter() - t0
        if r.t_arrival > now:
            time.sleep(r.t_arrival - now)
        with torch.cuda.stream(st):
            d_in = r.img.to(dev, non_blocking=True)
            out = api.snlm_denoise(d_in, r.S, r.K, r.h, r.profile, r.order, r.sigma, r.beta, stream=st)
            r.out.copy_(out, non_blocking=True)
        st.synchronize()
        r.t_done = time.perf_counter() - t0
        stats.latencies.append(r.latency())
        stats.sizes.append(r.shape[0])
        stats.images += 1
    stats.wall = time.perf_counter() - t0
    return stats



class NativeServer:
    """The library's own serving loop (snlm_server_* of include/snlm.h): the same
    admission, solo/batch launches over rotating streams and retirement as
    `Server`, run in C++ by the calling thread. mode "batched" is continuous
    batching; "plain" serves one request at a time through the per-image path (the
    per-request baseline, with the same host-side cost per request)."""

    def __init__(self, mode: str = "batched", mem_budget: int | None = None, streams: int = 4,
                 max_batch: int = 256, solo_pixels: int = 1024 * 1024, ctas_per_sm: int = 0):
        import torch

        self.mode = {"batched": 0, "plain": 1}[mode]
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info()
            mem_budget = min(free // 2, 16 << 30)
        self.cfg = (self.mode, int(mem_budget), int(streams), int(max_batch), int(solo_pixels), int(ctas_per_sm))

    def run(self, schedule, stats: ServeStats | None = None):
        stats = stats or ServeStats()
        prepare_outputs(schedule)
        mode, budget, streams, max_batch, solo, ctas = self.cfg
        handle = api.snlm_server_create(mode, budget, streams, max_batch, solo, ctas)
        try:
            ids = api.snlm_server_submit(handle, [dict(img=r.img, out=r.out, S=r.S, K=r.K, h=r.h, profile=r.profile,
                                                       order=r.order, sigma=r.sigma, beta=r.beta,
                                                       t_arrival=r.t_arrival) for r in schedule])
            api.snlm_server_drain(handle)
            for i, r in zip(ids, schedule):
                r.t_done, r.step = api.snlm_server_result(handle, i)
                stats.latencies.append(r.latency())
                stats.sizes.append(r.shape[0])
            st = api.snlm_server_get_stats(handle)
            stats.images, stats.steps, stats.max_batch = st["images"], st["launches"], st["max_batch"]
            stats.max_inflight, stats.max_used, stats.wall = st["max_inflight"], st["max_used_bytes"], st["wall_s"]
            stats.host_s = {"loop": st["host_busy_s"]}
            stats.loop = {"max_yield_ms": st["max_yield_s"] * 1e3, "max_iter_ms": st["max_iter_s"] * 1e3,
                          "yields_over_1ms": st["yields_over_1ms"]}
        finally:
            api.snlm_server_destroy(handle)
        return stats
