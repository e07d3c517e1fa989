"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: uint8 box patch distances are integers and must match bit for bit;
denoised float32 pixels must be within 1e-4 of the oracle on the [0, 255] scale;
float patch distances within a relative 2e-6 (a few float roundings of a sum of
at most 2K+1 non-negative terms); chained derivatives within a relative 1e-4.
"""
import math

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


@pytest.fixture(scope="module")
def api():
    from paper_1407_2343_gb300 import api

    return api


def to_dev(a, dev):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def np_of(t):
    return t.detach().cpu().numpy()


# ------------------------------------------------------------------ patch distances

@pytest.mark.parametrize("n,N,S,K", [(3, 1, 2, 1), (2, 7, 9, 3), (5, 100, 5, 2), (4, 233, 20, 5),
                                      (9, 1031, 10, 3), (1, 300, 25, 7), (2, 64, 0, 4), (3, 50, 8, 0)])
def test_patch_dist_u8_box_bit_exact(dev, api, orc, n, N, S, K):
    x = synth.signals(n, N, 30.0, seed=N + S, dtype="u8")
    got = np_of(api.snlm_patch_dist_1d(to_dev(x, dev), S, K, "box"))
    ref = orc.patch_dist_1d(x.astype(np.float64), S, K, "box")
    assert got.dtype == np.int32
    np.testing.assert_array_equal(got, ref.astype(np.int64))


@pytest.mark.parametrize("dtype,prof,K", [("f32", "box", 3), ("f16", "box", 5), ("f32", "gauss", 3),
                                           ("u8", "gauss", 5), ("f32", "gauss", 7)])
def test_patch_dist_float(dev, api, orc, dtype, prof, K):
    n, N, S = 6, 517, 12
    x = synth.signals(n, N, 25.0, seed=3, dtype=dtype)
    beta = K / 2.0
    got = np_of(api.snlm_patch_dist_1d(to_dev(x, dev), S, K, prof, beta)).astype(np.float64)
    ref = orc.patch_dist_1d(x.astype(np.float64), S, K, prof, beta)
    err = np.abs(got - ref) / np.maximum(ref, 1.0)
    assert err.max() <= 2e-6, err.max()


# ------------------------------------------------------------------ one 1-D pass

@pytest.mark.parametrize("dtype,prof,S,K", [("u8", "box", 10, 3), ("f32", "box", 20, 5), ("f16", "box", 7, 2),
                                             ("f32", "gauss", 10, 3), ("u8", "gauss", 15, 5), ("f32", "box", 3, 7)])
def test_nlm_1d_rows(dev, api, orc, dtype, prof, S, K):
    n, N, sigma = 11, 700, 25.0
    x = synth.signals(n, N, sigma, seed=S * 10 + K, dtype=dtype)
    beta = K / 2.0
    h = orc.default_h(sigma, K, prof, beta)
    got = np_of(api.snlm_nlm_1d(to_dev(x, dev), S, K, h, prof, beta))
    ref = orc.nlm_1d(x.astype(np.float64), S, K, h, prof, beta)
    assert np.abs(got - ref).max() <= TOL


def test_nlm_1d_strided_columns(dev, api, orc):
    import torch

    img = synth.noisy_image(300, 90, 20.0, seed=2, dtype="f32")
    S, K = 12, 3
    h = orc.default_h(20.0, K)
    t = to_dev(img, dev)
    got = np_of(api.snlm_nlm_1d(t.t(), S, K, h))          # lines = columns (stride W)
    ref = orc.nlm_1d(img.T.astype(np.float64), S, K, h)
    assert np.abs(got - ref).max() <= TOL
    # output written through a transposed view
    out = torch.empty((300, 90), dtype=torch.float32, device=dev)
    api.snlm_nlm_1d(t.t(), S, K, h, fhat=out.t())
    assert np.abs(np_of(out).T - ref).max() <= TOL


@pytest.mark.parametrize("dtype,prof,S,K", [("f32", "box", 10, 3), ("u8", "box", 20, 5), ("f32", "gauss", 8, 2),
                                             ("f16", "gauss", 12, 5)])
def test_nlm_1d_with_divergence(dev, api, orc, dtype, prof, S, K):
    import torch

    n, N, sigma = 7, 400, 20.0
    x = synth.signals(n, N, sigma, seed=5, dtype=dtype)
    beta = K / 2.0
    h = orc.default_h(sigma, K, prof, beta)
    rng = np.random.default_rng(1)
    din = rng.uniform(0.5, 1.5, size=(n, N))
    fh_ref, d_ref = orc.nlm_1d(x.astype(np.float64), S, K, h, prof, beta, delta_in=din)
    d_in = to_dev(din.astype(np.float32), dev)
    d_out = torch.empty_like(d_in)
    fh = api.snlm_nlm_1d(to_dev(x, dev), S, K, h, prof, beta, delta_in=d_in, delta_out=d_out)
    assert np.abs(np_of(fh) - fh_ref).max() <= TOL
    # relative to the float32 rounding of delta_in
    ref = d_ref * (din.astype(np.float32).astype(np.float64) / din)
    rel = np.abs(np_of(d_out) - ref) / np.maximum(np.abs(ref), 1e-3)
    assert rel.max() <= 1e-4, rel.max()
    # in place (delta_out aliasing delta_in)
    api.snlm_nlm_1d(to_dev(x, dev), S, K, h, prof, beta, delta_in=d_in, delta_out=d_in)
    assert np.array_equal(np_of(d_in), np_of(d_out))


# ------------------------------------------------------------------ whole images

def _oracle_ref(orc, img, S, K, h, prof, beta, order, sigma):
    out, info = orc.snlm(img.astype(np.float64), S, K, h, prof, beta, order=order, sigma=sigma)
    return out, info


@pytest.mark.parametrize("order", ["RC", "CR", "AVG", "SURE"])
@pytest.mark.parametrize("dtype", ["u8", "f16", "f32"])
def test_denoise_256(dev, api, orc, order, dtype):
    # the 256x256 synthetic scene (sigma = 20, S = 10, K = 3, box, h = sigma*sqrt(7))
    sigma, S, K = 20.0, 10, 3
    img = synth.noisy_image(256, 256, sigma, seed=0, dtype=dtype)
    h = orc.default_h(sigma, K)
    ref, info = _oracle_ref(orc, img, S, K, h, "box", 1.5, order, sigma)
    got = np_of(api.snlm_denoise(to_dev(img, dev), S, K, h, "box", order, sigma))
    err = np.abs(got - ref).max()
    assert err <= TOL, err


@pytest.mark.parametrize("H,W,S,K,prof", [(97, 131, 10, 3, "box"), (1, 77, 5, 2, "box"), (64, 1, 6, 1, "gauss"),
                                           (1, 1, 3, 2, "box"), (5, 9, 20, 5, "box"), (3, 300, 7, 7, "gauss"),
                                           (41, 33, 0, 3, "box"), (50, 70, 4, 0, "box"), (260, 240, 25, 5, "box")])
@pytest.mark.parametrize("order", ["RC", "SURE"])
def test_denoise_shapes(dev, api, orc, H, W, S, K, prof, order):
    sigma = 25.0
    img = synth.noisy_image(H, W, sigma, seed=H * W + S, dtype="f32")
    beta = max(K / 2.0, 0.5)
    h = orc.default_h(sigma, K, prof, beta)
    ref, _ = _oracle_ref(orc, img, S, K, h, prof, beta, order, sigma)
    got = np_of(api.snlm_denoise(to_dev(img, dev), S, K, h, prof, order, sigma, beta))
    assert np.abs(got - ref).max() <= TOL


def test_denoise_pitched_input_and_offset_output(dev, api, orc):
    import torch

    sigma, S, K = 20.0, 8, 2
    img = synth.noisy_image(120, 150, sigma, seed=4, dtype="u8")
    big = np.zeros((120, 173), np.uint8)
    big[:, 5:155] = img
    t = to_dev(big, dev)[:, 5:155]                       # pitch 173, unaligned start
    h = orc.default_h(sigma, K)
    buf = torch.empty(120 * 150 + 1, dtype=torch.float32, device=dev)
    out = buf[1:].view(120, 150)                         # 4-byte aligned, not 16-byte aligned
    for order in ("RC", "SURE"):
        ref, _ = _oracle_ref(orc, img, S, K, h, "box", 1.0, order, sigma)
        api.snlm_denoise(t, S, K, h, "box", order, sigma, out=out)
        assert np.abs(np_of(out) - ref).max() <= TOL


@pytest.mark.parametrize("sigma", [10.0, 20.0, 30.0, 50.0])
def test_denoise_512_sweep(dev, api, orc, sigma):
    # 512x512 float32, S = 10, K in {2, 3, 5}, box and Gaussian (beta = K/2), all orders
    import torch

    img = synth.noisy_image(512, 512, sigma, seed=int(sigma), dtype="f32")
    t = to_dev(img, dev)
    worst = 0.0
    for prof in ("box", "gauss"):
        for K in (2, 3, 5):
            beta = K / 2.0
            h = orc.default_h(sigma, K, prof, beta)
            parts = orc.snlm_parts(img.astype(np.float64), 10, K, h, prof, beta)
            sure_ref, info = orc.snlm(img.astype(np.float64), 10, K, h, prof, beta, order="SURE", sigma=sigma)
            refs = {"RC": parts["frc"], "CR": parts["fcr"], "AVG": 0.5 * (parts["frc"] + parts["fcr"]),
                    "SURE": sure_ref}
            for order, ref in refs.items():
                inf = torch.zeros(10, dtype=torch.float64, device=dev)
                got = np_of(api.snlm_denoise_ws(t, 10, K, h, prof, order, sigma, beta, info=inf))
                err = float(np.abs(got - ref).max())
                worst = max(worst, err)
                assert err <= TOL, (prof, K, order, err)
                if order == "SURE":
                    gi = np_of(inf)
                    assert gi[0] == pytest.approx(info["theta1"], abs=1e-5)
                    assert gi[1] == pytest.approx(info["theta2"], abs=1e-5)
                    assert gi[7] == pytest.approx(info["sum_d1"], rel=1e-5)
                    assert gi[8] == pytest.approx(info["sum_d2"], rel=1e-5)


def test_denoise_invariants(dev, api, orc):
    import torch

    # constant image unchanged (RC/CR/AVG); S = 0 is the identity
    c = np.full((70, 90), 133.0, np.float32)
    for order in ("RC", "CR", "AVG"):
        got = np_of(api.snlm_denoise(to_dev(c, dev), 10, 3, 30.0, "box", order))
        assert np.array_equal(got, c)
    img = synth.noisy_image(60, 80, 20.0, seed=1, dtype="f32")
    assert np.array_equal(np_of(api.snlm_denoise(to_dev(img, dev), 0, 3, 30.0)), img)
    # h -> 0: identity; h -> infinity: separable window mean
    u8 = synth.noisy_image(60, 80, 20.0, seed=1, dtype="u8")
    assert np.array_equal(np_of(api.snlm_denoise(to_dev(u8, dev), 6, 2, 1e-18)), u8.astype(np.float32))
    ref, _ = orc.snlm(u8.astype(np.float64), 6, 2, 1e30, order="RC")
    got = np_of(api.snlm_denoise(to_dev(u8, dev), 6, 2, 1e30))
    assert np.abs(got - ref).max() <= TOL
    # output within the range of the input (each pass is a convex combination)
    got = np_of(api.snlm_denoise(to_dev(u8, dev), 10, 3, 50.0, "box", "AVG"))
    assert got.min() >= u8.min() - 1e-3 and got.max() <= u8.max() + 1e-3
    # deterministic: bitwise identical repeat, SURE included
    t = to_dev(img, dev)
    a = np_of(api.snlm_denoise(t, 10, 3, 40.0, "box", "SURE", 20.0))
    b = np_of(api.snlm_denoise(t, 10, 3, 40.0, "box", "SURE", 20.0))
    assert np.array_equal(a, b)


def test_denoise_host_entry_point(dev, api, orc):
    import torch

    img = synth.noisy_image(130, 170, 20.0, seed=6, dtype="u8")
    h = orc.default_h(20.0, 3)
    ref, _ = orc.snlm(img.astype(np.float64), 10, 3, h, order="SURE", sigma=20.0)
    out = api.snlm_denoise_host(img, 10, 3, h, "box", "SURE", 20.0)
    assert np.abs(out - ref).max() <= TOL
    pinned = torch.from_numpy(img).pin_memory()
    out2 = api.snlm_denoise_host(pinned, 10, 3, h, "box", "SURE", 20.0)
    assert np.array_equal(out, out2)


def test_pipelined_host_entry_point_equals_single_calls(dev, api, orc):
    import ctypes

    import torch
    from paper_1407_2343_gb300 import _lib

    # five images of different content: pinned CPU tensors and pageable arrays mixed;
    # every result equals the synchronous single-image call bit for bit
    sigma, S, K = 20.0, 10, 3
    h = orc.default_h(sigma, K)
    imgs = [synth.noisy_image(140, 190, sigma, seed=20 + i, dtype="u8") for i in range(5)]
    hosts = [torch.from_numpy(im).pin_memory() if i % 2 == 0 else im for i, im in enumerate(imgs)]
    outs = [torch.empty((140, 190), dtype=torch.float32).pin_memory() if i % 2 == 0 else None for i in range(5)]
    outs = [o if o is not None else np.empty((140, 190), np.float32) for o in outs]
    got = api.snlm_denoise_host_many(hosts, S, K, h, "box", "SURE", sigma, outs=outs)
    for i, im in enumerate(imgs):
        single = api.snlm_denoise_host(im, S, K, h, "box", "SURE", sigma)
        g = got[i].numpy() if isinstance(got[i], torch.Tensor) else got[i]
        assert np.array_equal(g, single), i
    ref, _ = orc.snlm(imgs[3].astype(np.float64), S, K, h, order="SURE", sigma=sigma)
    assert np.abs(got[3] - ref).max() <= TOL
    assert api.snlm_denoise_host_many([], S, K, h, "box", "SURE", sigma) == []
    with pytest.raises(ValueError):
        api.snlm_denoise_host_many([imgs[0], imgs[1][:, :100]], S, K, h, "box", "SURE", sigma)
    # C level: a NULL entry or a negative count is an argument error and writes nothing
    lib = _lib.load()
    out = np.full((140, 190), 7.0, np.float32)
    iarr = (ctypes.c_void_p * 2)(imgs[0].ctypes.data, None)
    oarr = (ctypes.c_void_p * 2)(out.ctypes.data, out.ctypes.data)
    assert lib.snlm_denoise_host_many(iarr, oarr, 2, api.U8, 140, 190, 190, S, K, h, 0, 3, sigma, 0.0,
                                      None) == api.ERR_ARG
    assert lib.snlm_denoise_host_many(iarr, oarr, -1, api.U8, 140, 190, 190, S, K, h, 0, 3, sigma, 0.0,
                                      None) == api.ERR_ARG
    assert (out == 7.0).all()


def test_argument_errors_leave_output_untouched(dev, api):
    import ctypes

    import torch
    from paper_1407_2343_gb300 import _lib

    lib = _lib.load()
    img = torch.zeros((16, 16), dtype=torch.uint8, device=dev)
    out = torch.full((16, 16), 7.0, device=dev)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.snlm_denoise(p(img), 0, 16, 16, 16, -1, 3, 10.0, 0, 0, 0.0, 0.0, p(out), s) == api.ERR_ARG
    assert lib.snlm_denoise(p(img), 0, 16, 16, 16, 5, 8, 10.0, 0, 0, 0.0, 0.0, p(out), s) == api.ERR_UNSUPPORTED
    assert lib.snlm_denoise(p(img), 0, 16, 16, 16, 5, 3, 0.0, 0, 0, 0.0, 0.0, p(out), s) == api.ERR_ARG
    assert lib.snlm_denoise(p(img), 0, 16, 16, 16, 5, 3, float("nan"), 0, 0, 0.0, 0.0, p(out), s) == api.ERR_ARG
    assert lib.snlm_denoise(p(img), 9, 16, 16, 16, 5, 3, 10.0, 0, 0, 0.0, 0.0, p(out), s) == api.ERR_ARG
    assert lib.snlm_denoise(p(img), 0, 16, 16, 8, 5, 3, 10.0, 0, 0, 0.0, 0.0, p(out), s) == api.ERR_ARG
    assert lib.snlm_denoise(p(img), 0, 16, 16, 16, 5, 3, 10.0, 0, 3, -1.0, 0.0, p(out), s) == api.ERR_ARG
    assert lib.snlm_denoise(None, 0, 16, 16, 16, 5, 3, 10.0, 0, 0, 0.0, 0.0, p(out), s) == api.ERR_ARG
    host = np.zeros((16, 16), np.float32)
    assert lib.snlm_denoise(p(img), 0, 16, 16, 16, 5, 3, 10.0, 0, 0, 0.0, 0.0,
                            ctypes.c_void_p(host.ctypes.data), s) == api.ERR_ARG
    small_ws = torch.empty(64, dtype=torch.uint8, device=dev)
    assert lib.snlm_denoise_ws(p(img), 0, 16, 16, 16, 5, 3, 10.0, 0, 0, 0.0, 0.0, p(out), p(small_ws), 64,
                               None, s) == api.ERR_ARG
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())


def test_full_size_whole_image_parity(dev, api, orc):
    # 4096x4096 uint8, S = 20, K = 5, box, sigma = 30: the benchmark's launch
    # configuration, compared with the oracle over the whole image. RC and CR
    # element by element, the SURE output element by element, and the SURE system
    # of Alg. 4: theta and the seven sums of Eqs. (19) and (25).
    import torch

    H = W = 4096
    S, K, sigma = 20, 5, 30.0
    img = synth.noisy_image(H, W, sigma, seed=0, dtype="u8")
    t = to_dev(img, dev)
    h = orc.default_h(sigma, K)
    f = img.astype(np.float64)
    for order in ("RC", "CR"):
        got = np_of(api.snlm_denoise(t, S, K, h, "box", order)).astype(np.float64)
        ref, _ = orc.snlm(f, S, K, h, "box", order=order)
        err = float(np.abs(got - ref).max())
        assert err <= TOL, (order, err)
    info = torch.zeros(10, dtype=torch.float64, device=dev)
    sure = np_of(api.snlm_denoise_ws(t, S, K, h, "box", "SURE", sigma, info=info)).astype(np.float64)
    gi = np_of(info)
    ref, ri = orc.snlm(f, S, K, h, "box", order="SURE", sigma=sigma)
    err = float(np.abs(sure - ref).max())
    assert err <= TOL, err
    assert abs(gi[0] - ri["theta1"]) <= 1e-6 and abs(gi[1] - ri["theta2"]) <= 1e-6, (gi[:2], ri)
    for k, name in enumerate(["A11", "A12", "A22", "sum_f_frc", "sum_f_fcr", "sum_d1", "sum_d2"]):
        assert gi[2 + k] == pytest.approx(ri[name], rel=1e-5), name
    # patch distances of the first rows, bit exact
    d = np_of(api.snlm_patch_dist_1d(t[:4], S, K, "box"))
    np.testing.assert_array_equal(d, orc.patch_dist_1d(img[:4].astype(np.float64), S, K, "box").astype(np.int64))


def test_preload_loads_every_kernel(dev, api):
    import time

    assert api.snlm_preload() == api.KERNEL_COUNT
    t0 = time.perf_counter()
    assert api.snlm_preload() == api.KERNEL_COUNT      # already loaded: lookups only
    assert time.perf_counter() - t0 < 0.5
