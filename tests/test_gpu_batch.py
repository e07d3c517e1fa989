"""Batched persistent launches (snlm_batch_*) against the FP64 oracle and the
per-image entry point.

Every batched output, SURE included, is compared with the oracle's Alg. 4 on the
same stored samples within the 1e-4 tolerance. Against snlm_denoise, RC, CR and
AVG results must be equal bit for bit (each unit runs the same code on the same
data); SURE results within 1e-4 (the per-image sums are reduced in a different
fixed order, so theta may differ in its last bits).
"""
import numpy as np
import pytest

from paper_1407_2343_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def dev():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_2343_gb300 import _lib, build

    build.build()
    _lib.load()
    return torch.device("cuda:0")


def make_requests(dev, specs):
    import torch

    from paper_1407_2343_gb300 import api

    reqs = []
    for i, s in enumerate(specs):
        img = torch.from_numpy(synth.noisy_image(s["H"], s["W"], s["sigma"], seed=100 + i, dtype=s["dtype"])).to(dev)
        out = torch.full((s["H"], s["W"]), float("nan"), dtype=torch.float32, device=dev)
        beta = s.get("beta", s["K"] / 2.0)
        h = api.snlm_default_h(s["sigma"], s["K"], s.get("profile", "box"), beta)
        reqs.append(dict(img=img, out=out, S=s["S"], K=s["K"], h=h, profile=s.get("profile", "box"),
                         order=s.get("order", "RC"), sigma=s["sigma"], beta=beta))
    return reqs


def reference(r):
    from paper_1407_2343_gb300 import api

    return api.snlm_denoise(r["img"], r["S"], r["K"], r["h"], r["profile"], r["order"], r["sigma"], r["beta"])


MIXED = [dict(H=64, W=90, dtype="u8", sigma=20, S=5, K=2),
         dict(H=130, W=77, dtype="f16", sigma=30, S=10, K=3, order="CR"),
         dict(H=257, W=300, dtype="u8", sigma=15, S=15, K=5, order="AVG"),
         dict(H=100, W=100, dtype="f32", sigma=25, S=7, K=3, order="SURE"),
         dict(H=33, W=500, dtype="u8", sigma=40, S=10, K=2, profile="gauss"),
         dict(H=512, W=64, dtype="f16", sigma=10, S=20, K=5, order="SURE", profile="gauss"),
         dict(H=1, W=200, dtype="f32", sigma=20, S=6, K=1),
         dict(H=90, W=1, dtype="u8", sigma=20, S=3, K=2, order="AVG"),
         dict(H=70, W=80, dtype="u8", sigma=20, S=0, K=3),
         dict(H=200, W=180, dtype="u8", sigma=35, S=12, K=5)]


def expected_classes(specs):
    """One class per (dependency level, pass variant, K), and the solve and the
    combination jobs of SURE in classes of their own levels. A pass over the stored
    image uses the running sums (uint8, box), the block sums (other storage, box) or
    the Gaussian taps; a pass over a float intermediate the block sums or the
    Gaussian taps; SURE passes are variants of their own. Levels: the passes over
    the image 0, the pass over the first intermediate 1, the last pass of AVG and
    SURE (which also reads the other order's result) 2, the solve 3, the combination
    4."""
    keys = set()
    for s in specs:
        gauss = s.get("profile", "box") == "gauss"
        order = s.get("order", "RC")
        sure = order == "SURE"
        img = "fir" if gauss else ("slide" if s["dtype"] == "u8" else "block")
        f32 = "fir" if gauss else "block"
        keys.add((0, img, sure, s["K"]))
        keys.add((2 if order in ("AVG", "SURE") else 1, f32, sure, s["K"]))
        if order in ("AVG", "SURE"):
            keys.add((1, f32, sure, s["K"]))
        if sure:
            keys.add((3, "solve"))
            keys.add((4, "combine"))
    return len(keys)


def oracle_out(r):
    """Alg. 4 of the FP64 oracle on the request's stored samples."""
    import oracle

    oracle.build()
    f = r["img"].cpu().numpy().astype(np.float64)
    out, _ = oracle.snlm(f, r["S"], r["K"], r["h"], r["profile"], r["beta"], order=r["order"], sigma=r["sigma"])
    return out


def check(reqs, with_oracle=True):
    for r in reqs:
        ref = reference(r).cpu().numpy()
        got = r["out"].cpu().numpy()
        if r["order"] == "SURE":
            assert np.abs(got - ref).max() <= TOL, (r["img"].shape, r["order"])
        else:
            assert np.array_equal(got, ref), (r["img"].shape, r["order"], np.abs(got - ref).max())
        if with_oracle:
            err = float(np.abs(got.astype(np.float64) - oracle_out(r)).max())
            assert err <= TOL, (r["img"].shape, r["order"], r["profile"], err)


def test_batch_matches_per_image(dev):
    import torch

    from paper_1407_2343_gb300 import api
    from paper_1407_2343_gb300.batch import Batch

    reqs = make_requests(dev, MIXED)
    b = Batch(reqs)
    info = b.info()
    assert info["classes"] == expected_classes(MIXED) and info["jobs"] > len(reqs)
    b.run()
    torch.cuda.synchronize()
    assert b.status() == api.OK
    check(reqs)
    b.close()


@pytest.mark.parametrize("ctas,order", [(1, 0), (2, 1), (3, 2), (0, 0)])
def test_batch_launch_parameters_do_not_change_results(dev, ctas, order):
    import torch

    from paper_1407_2343_gb300.batch import Batch

    reqs = make_requests(dev, MIXED[:6])
    b = Batch(reqs, ctas_per_sm=ctas, queue_order=order)
    b.run()
    torch.cuda.synchronize()
    assert b.status() == 0
    check(reqs)
    b.close()


def test_batch_graph_replay(dev):
    import torch

    from paper_1407_2343_gb300.batch import Batch

    reqs = make_requests(dev, MIXED)
    b = Batch(reqs)
    b.capture()
    for _ in range(3):
        for r in reqs:
            r["out"].fill_(float("nan"))
        b.run()
        torch.cuda.synchronize()
        assert b.status() == 0
        check(reqs)
    b.close()


def test_batch_uneven_workload_recipe(dev):
    # 40 images drawn from the uneven batch recipe (sides 64..1024, u8/f16, S in
    # {5,10,15}, K in {2,3,5}, box), the four orders of Alg. 4 in turn, each
    # against the per-image path and the oracle
    import torch

    from paper_1407_2343_gb300 import api
    from paper_1407_2343_gb300.batch import Batch

    specs = synth.batch_specs(40, seed=1)
    for i, sp in enumerate(specs):          # every order of Alg. 4 in the mix
        sp["order"] = ("RC", "CR", "AVG", "SURE")[i % 4]
    reqs = make_requests(dev, specs)
    b = Batch(reqs, queue_order=1)
    b.capture()
    b.run()
    torch.cuda.synchronize()
    assert b.status() == api.OK
    check(reqs)
    b.close()


def test_batch_bounded_wait_reports_timeout(dev):
    # host-side fault injection: one job's dependency can never be satisfied; the
    # waits give up after 20 ms, the run reports SNLM_ERR_TIMEOUT, and the device
    # stays usable.
    import torch

    from paper_1407_2343_gb300 import api
    from paper_1407_2343_gb300.batch import Batch

    reqs = make_requests(dev, MIXED[:3])
    # the plan's last job (the highest dependency level) has a dependency to break
    probe = Batch(reqs)
    last = probe.info()["jobs"] - 1
    probe.close()
    b = Batch(reqs, spin_limit_us=20000, fail_job=last)
    word = torch.full((1,), -7, dtype=torch.int32).pin_memory()
    st = torch.cuda.current_stream()
    b.run(st)
    api.snlm_batch_plan_status_async(b.plan, word, st)    # the same report without waiting
    torch.cuda.synchronize()
    assert int(word[0]) != 0
    assert b.status() == api.ERR_TIMEOUT
    b.close()
    # the context still works
    reqs2 = make_requests(dev, MIXED[:2])
    b2 = Batch(reqs2)
    b2.run(st)
    api.snlm_batch_plan_status_async(b2.plan, word, st)
    torch.cuda.synchronize()
    assert int(word[0]) == 0
    assert b2.status() == api.OK
    check(reqs2)
    b2.close()


def test_batch_rejects_bad_requests(dev):
    import torch

    from paper_1407_2343_gb300 import api
    from paper_1407_2343_gb300.batch import Batch

    reqs = make_requests(dev, MIXED[:2])
    reqs[1]["K"] = 0
    with pytest.raises(api.SnlmError) as e:
        Batch(reqs)
    assert e.value.status == api.ERR_UNSUPPORTED
    reqs[1]["K"] = 9
    with pytest.raises(api.SnlmError):
        Batch(reqs)
    reqs[1]["K"] = 2
    reqs[1]["S"] = -1
    with pytest.raises(api.SnlmError) as e:
        Batch(reqs)
    assert e.value.status == api.ERR_ARG
    torch.cuda.synchronize()


def test_autotune_caches_a_choice(dev, tmp_path):
    from paper_1407_2343_gb300.batch import autotune

    reqs = make_requests(dev, MIXED[:5])
    cache = str(tmp_path / "tune.json")
    cands = [dict(ctas_per_sm=1, queue_order=0), dict(ctas_per_sm=0, queue_order=1)]
    cfg, table = autotune(reqs, candidates=cands, reps=2, cache_path=cache)
    assert cfg in [{k: c[k] for k in ("ctas_per_sm", "queue_order")} for c in cands]
    assert len(table) == 2 and all(t["ms"] > 0 for t in table)
    cfg2, _ = autotune(reqs, candidates=cands, reps=2, cache_path=cache)
    assert cfg2 == cfg
