"""The continuous-batching service (the Python loop `Server` and the library's own
loop `NativeServer`): schedule generation (CPU), and on the GPU the result of every
request alone equals its result in the mix, every served result of a mixed schedule
(sizes up to 512^2, every order, both profiles, u8 and f16 storage) is within 1e-4
of the FP64 oracle, launches overlap, admission under a memory cap, the plain (one
request at a time) mode, and rejection of a request larger than the whole budget."""
import math

import numpy as np
import pytest

from paper_1407_2343_gb300 import serve

TOL = 1e-4


def test_schedule_statistics():
    reqs = serve.make_schedule(400, rate=1000.0, seed=3, sizes=(16, 32, 48), weights=(0.5, 0.3, 0.2), pin=False)
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1e-3) < 0.2e-3          # Poisson at 1000/s
    frac = np.mean([r.shape[0] == 16 for r in reqs])
    assert abs(frac - 0.5) < 0.08
    for r in reqs:
        assert r.S in (5, 10, 15, 20) and r.K in (2, 3, 5)
        assert r.profile in ("box", "gauss") and r.order in ("RC", "CR", "AVG", "SURE")
        if r.profile == "box":
            assert r.h == pytest.approx(r.sigma * math.sqrt(2 * r.K + 1), rel=1e-6)


def test_stats_split_latencies_by_image_size():
    st = serve.ServeStats(latencies=[0.001, 0.003, 0.002, 0.010, 0.030], sizes=[128, 128, 128, 4096, 4096],
                          wall=1.0, images=5)
    by = st.summary()["by_size"]
    assert set(by) == {"128", "4096"}
    assert by["128"]["n"] == 3 and by["128"]["p50_ms"] == pytest.approx(2.0)
    assert by["4096"]["n"] == 2 and by["4096"]["p99_ms"] == pytest.approx(29.8)
    # a run that recorded no sizes reports none
    assert serve.ServeStats(latencies=[0.001], wall=1.0, images=1).summary()["by_size"] == {}


@pytest.fixture(scope="module")
def dev():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_2343_gb300 import _lib, build

    build.build()
    _lib.load()
    return torch.device("cuda:0")


def oracle_out(r):
    """Alg. 4 of the FP64 oracle on the request's stored samples."""
    import oracle

    oracle.build()
    f = r.img.numpy().astype(np.float64)
    out, _ = oracle.snlm(f, r.S, r.K, r.h, r.profile, r.beta, order=r.order, sigma=r.sigma)
    return out


def alone(r, dev):
    from paper_1407_2343_gb300 import api

    out = api.snlm_denoise(r.img.to(dev), r.S, r.K, r.h, r.profile, r.order, r.sigma, r.beta)
    return out.cpu().numpy()


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix(dev):
    reqs = serve.make_schedule(40, rate=4000.0, seed=1, sizes=(128, 256, 512), weights=(0.5, 0.3, 0.2))
    stats = serve.Server(dev).run(reqs)
    assert stats.images == len(reqs)
    assert stats.max_batch > 1                         # requests were batched together
    for r in reqs:
        ref = alone(r, dev)
        got = r.out.numpy()
        if r.order == "SURE":
            assert np.abs(got - ref).max() <= TOL
        else:
            assert np.array_equal(got, ref), (r.rid, r.order)
    s = stats.summary()
    assert s["p50_ms"] > 0 and s["p99_ms"] >= s["p50_ms"]


@pytest.mark.gpu
def test_admission_under_a_memory_cap(dev):
    from paper_1407_2343_gb300 import api

    reqs = serve.make_schedule(12, rate=10000.0, seed=2, sizes=(256,), weights=(1.0,))
    cap = max(serve._footprint(r) for r in reqs) * 2 + 1
    stats = serve.Server(dev, mem_budget=cap).run(reqs)
    assert stats.images == 12
    assert stats.max_used <= cap                       # never more than the cap admitted
    assert stats.steps >= 4                            # so the requests went through in several steps
    for r in reqs[:4]:
        ref = alone(r, dev)
        tol = TOL if r.order == "SURE" else 0.0
        assert np.abs(r.out.numpy() - ref).max() <= tol
    big = serve.make_schedule(1, rate=1.0, seed=4, sizes=(512,), weights=(1.0,))
    with pytest.raises(ValueError):
        serve.Server(dev, mem_budget=1024).run(big)
    assert api.snlm_version() >= 100


@pytest.mark.gpu
def test_native_server_results_alone_equal_results_in_the_mix(dev):
    # arrivals faster than the GPU serves them (a burst), so that requests queue up and
    # share batch launches with each other
    reqs = serve.make_schedule(48, rate=50000.0, seed=7, sizes=(128, 256, 512, 1024), weights=(0.4, 0.3, 0.2, 0.1))
    stats = serve.NativeServer("batched").run(reqs)
    assert stats.images == len(reqs)
    assert stats.max_batch > 1                         # small requests shared launches
    assert stats.max_inflight > 1                      # launches overlapped on the device
    for r in reqs:
        ref = alone(r, dev)
        got = r.out.numpy()
        if r.order == "SURE":
            assert np.abs(got - ref).max() <= TOL
        else:
            assert np.array_equal(got, ref), (r.rid, r.order)
        assert r.t_done >= r.t_arrival
    s = stats.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["batched", "plain"])
def test_served_results_match_the_oracle(dev, mode):
    # a burst of mixed requests (128^2 to 512^2; S, K, profile, order and storage
    # drawn per request), served by the native loop, every result against the oracle
    reqs = serve.make_schedule(32, rate=50000.0, seed=11, sizes=(128, 256, 512), weights=(0.4, 0.35, 0.25))
    stats = serve.NativeServer(mode).run(reqs)
    assert stats.images == len(reqs)
    if mode == "batched":
        assert stats.max_batch > 1
    assert {r.order for r in reqs} == {"RC", "CR", "AVG", "SURE"}
    for r in reqs:
        err = float(np.abs(r.out.numpy().astype(np.float64) - oracle_out(r)).max())
        assert err <= TOL, (r.rid, r.shape, r.order, r.profile, r.S, r.K, err)


@pytest.mark.gpu
def test_native_plain_mode_serves_one_at_a_time(dev):
    reqs = serve.make_schedule(10, rate=1e6, seed=8, sizes=(128, 256), weights=(0.5, 0.5))
    stats = serve.NativeServer("plain").run(reqs)
    assert stats.images == 10 and stats.max_batch == 1 and stats.max_inflight == 1
    # the loop's own timing record and the per-size split of the latencies
    assert set(stats.loop) == {"max_yield_ms", "max_iter_ms", "yields_over_1ms"}
    assert stats.loop["max_iter_ms"] >= 0.0 and stats.loop["yields_over_1ms"] >= 0
    by = stats.summary()["by_size"]
    assert sum(v["n"] for v in by.values()) == 10 and set(by) <= {"128", "256"}
    for r in reqs[:4]:
        ref = alone(r, dev)
        tol = TOL if r.order == "SURE" else 0.0
        assert np.abs(r.out.numpy() - ref).max() <= tol


@pytest.mark.gpu
def test_native_server_admission_under_a_memory_cap(dev):
    from paper_1407_2343_gb300 import api

    reqs = serve.make_schedule(12, rate=1e6, seed=2, sizes=(256,), weights=(1.0,))
    cap = max(serve._footprint(r) for r in reqs) * 3
    stats = serve.NativeServer("batched", mem_budget=cap).run(reqs)
    assert stats.images == 12
    assert 0 < stats.max_used <= cap
    assert stats.steps >= 3                            # memory forced several launches
    for r in reqs[:4]:
        ref = alone(r, dev)
        tol = TOL if r.order == "SURE" else 0.0
        assert np.abs(r.out.numpy() - ref).max() <= tol
    big = serve.make_schedule(1, rate=1.0, seed=4, sizes=(512,), weights=(1.0,))
    with pytest.raises(api.SnlmError) as e:
        serve.NativeServer("batched", mem_budget=1 << 20).run(big)
    assert e.value.status == api.ERR_NOMEM
