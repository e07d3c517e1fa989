"""Parity of the recursive Gaussian profile (SNLM_GAUSS_IIR) with the FP64 oracle.

The CUDA path runs the Young-van Vliet recursion in float32 as a scan over the
lanes of a warp (each lane recurs over its 16 positions from rest, the end states
are combined across lanes by shuffles, and each lane recurs again from the state
entering its run) and truncates the filter's history where its causal response
falls below 1e-9 of its peak; the oracle recurs sequentially in FP64 from rest far
outside the line. Tolerances from that arithmetic:
  distances   |gpu - oracle| <= 1e-5 * (largest distance of the line) + 1e-5 * oracle:
              float32 rounding of the recursion grows with the state it carries
              (a few 1e-7 of the line's largest value per pass, amplified by
              1/B of the recursion: about 15 at beta = 3.5);
  pixels      1e-4 max-abs on the [0, 255] scale, as for every float32 output.
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


@pytest.fixture(scope="module")
def api():
    from paper_1407_2343_gb300 import api

    return api


def to_dev(a, dev):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def np_of(t):
    return t.detach().cpu().numpy()


def _dist_close(got, ref):
    scale = ref.reshape(ref.shape[0], -1).max(axis=1)[:, None, None]
    err = np.abs(got - ref) - (1e-5 * np.maximum(scale, 1.0) + 1e-5 * ref)
    assert err.max() <= 0.0, float((np.abs(got - ref) / np.maximum(scale, 1.0)).max())


@pytest.mark.parametrize("n,N,S,beta,dtype", [(3, 1, 2, 1.0, "f32"), (2, 7, 9, 1.5, "u8"), (5, 100, 5, 0.5, "f32"),
                                               (4, 233, 20, 2.5, "u8"), (9, 1031, 10, 1.5, "f16"),
                                               (2, 700, 25, 3.5, "f32"), (2, 64, 0, 2.0, "u8"),
                                               (3, 1500, 40, 2.5, "u8"), (1, 383, 128, 3.5, "f32")])
def test_patch_dist(dev, api, orc, n, N, S, beta, dtype):
    x = synth.signals(n, N, 30.0, seed=N + S, dtype=dtype)
    got = np_of(api.snlm_patch_dist_1d(to_dev(x, dev), S, 5, "gauss_iir", beta))
    assert got.dtype == np.float32 and got.shape == (n, N, 2 * S + 1)
    got = got.astype(np.float64)
    ref = orc.patch_dist_1d(x.astype(np.float64), S, 5, "gauss_iir", beta)
    _dist_close(got, ref)
    assert np.all(got[:, :, S] == 0.0)


@pytest.mark.parametrize("dtype,S,beta,sigma", [("u8", 10, 1.5, 20.0), ("f32", 20, 2.5, 10.0), ("f16", 7, 1.0, 30.0),
                                                 ("u8", 15, 2.5, 50.0), ("f32", 3, 3.5, 25.0), ("u8", 20, 3.5, 10.0)])
def test_nlm_1d_rows(dev, api, orc, dtype, S, beta, sigma):
    n, N = 11, 700
    x = synth.signals(n, N, sigma, seed=S * 10 + int(beta * 2), dtype=dtype)
    h = orc.default_h(sigma, 5, "gauss_iir", beta)
    assert api.snlm_default_h(sigma, 5, "gauss_iir", beta) == pytest.approx(h, rel=1e-6)
    got = np_of(api.snlm_nlm_1d(to_dev(x, dev), S, 5, h, "gauss_iir", beta))
    ref = orc.nlm_1d(x.astype(np.float64), S, 5, h, "gauss_iir", beta)
    assert np.abs(got - ref).max() <= TOL


def test_nlm_1d_strided_columns(dev, api, orc):
    import torch

    sigma, S, beta = 20.0, 12, 2.0
    img = synth.noisy_image(300, 45, sigma, seed=3, dtype="f32")
    h = orc.default_h(sigma, 4, "gauss_iir", beta)
    t = to_dev(img, dev)
    out = torch.zeros_like(t)
    from paper_1407_2343_gb300 import _lib

    lib = _lib.load()
    rc = lib.snlm_nlm_1d(t.data_ptr(), 2, 45, 300, 1, 45, S, 4, h, 2, beta, out.data_ptr(), 1, 45, None, None, None)
    assert rc == 0
    torch.cuda.synchronize()
    ref = orc.nlm_1d(img.T.astype(np.float64), S, 4, h, "gauss_iir", beta).T
    assert np.abs(np_of(out) - ref).max() <= TOL


@pytest.mark.parametrize("order", ["RC", "CR", "AVG", "SURE"])
@pytest.mark.parametrize("dtype", ["u8", "f16", "f32"])
def test_denoise_256(dev, api, orc, order, dtype):
    # the 256x256 scene of the small configuration (sigma = 20, S = 10) with the
    # recursive profile at beta = K/2 = 1.5
    sigma, S, K, beta = 20.0, 10, 3, 1.5
    img = synth.noisy_image(256, 256, sigma, seed=0, dtype=dtype)
    h = orc.default_h(sigma, K, "gauss_iir", beta)
    ref, _ = orc.snlm(img.astype(np.float64), S, K, h, "gauss_iir", beta, order=order, sigma=sigma)
    got = np_of(api.snlm_denoise(to_dev(img, dev), S, K, h, "gauss_iir", order, sigma, beta))
    assert np.abs(got - ref).max() <= TOL


@pytest.mark.parametrize("sigma,S,K,dtype", [(10.0, 10, 2, "f32"), (20.0, 10, 3, "u8"), (30.0, 10, 5, "f16"),
                                             (50.0, 20, 7, "u8"), (25.0, 0, 3, "f32")])
def test_sure_order_theta_and_sums(dev, api, orc, sigma, S, K, dtype):
    # Alg. 4 in the SURE order with the recursive profile: the divergence of Eq. (24)
    # with the profile's centre weight and its patch term over the whole window
    # (reading R17), theta of Eqs. (19), (25) and the seven sums against the oracle
    import torch

    beta = K / 2.0
    img = synth.noisy_image(200, 230, sigma, seed=int(sigma) + S + K, dtype=dtype)
    h = orc.default_h(sigma, K, "gauss_iir", beta)
    ref, ri = orc.snlm(img.astype(np.float64), S, K, h, "gauss_iir", beta, order="SURE", sigma=sigma)
    info = torch.zeros(10, dtype=torch.float64, device=dev)
    got = np_of(api.snlm_denoise_ws(to_dev(img, dev), S, K, h, "gauss_iir", "SURE", sigma, beta, info=info))
    gi = np_of(info)
    assert np.abs(got - ref).max() <= TOL
    assert abs(gi[0] - ri["theta1"]) <= 1e-5 and abs(gi[1] - ri["theta2"]) <= 1e-5, (gi[:2], ri)
    for k, name in enumerate(["A11", "A12", "A22", "sum_f_frc", "sum_f_fcr"]):
        assert gi[2 + k] == pytest.approx(ri[name], rel=1e-5), name
    for k, name in ((7, "sum_d1"), (8, "sum_d2")):
        assert gi[k] == pytest.approx(ri[name], rel=1e-4, abs=1e-2), name


def test_sure_order_in_row_bands(dev, api, orc):
    # the banded SURE exchange with the recursive profile: bands widened by its reach
    import torch

    from paper_1407_2343_gb300 import shard

    sigma, S, K, beta = 25.0, 10, 5, 2.5
    img = synth.noisy_image(300, 180, sigma, seed=3, dtype="u8")
    h = orc.default_h(sigma, K, "gauss_iir", beta)
    t = to_dev(img, dev)
    whole = api.snlm_denoise(t, S, K, h, "gauss_iir", "SURE", sigma, beta)
    ref, ri = orc.snlm(img.astype(np.float64), S, K, h, "gauss_iir", beta, order="SURE", sigma=sigma)
    for n in (2, 3):
        banded, theta = shard.denoise_bands(t, S, K, h, "gauss_iir", "SURE", beta, n_bands=n, sigma=sigma)
        torch.cuda.synchronize()
        assert float((banded - whole).abs().max()) <= TOL
        assert np.abs(np_of(banded) - ref).max() <= TOL
        assert abs(theta[0] - ri["theta1"]) <= 1e-5 and abs(theta[1] - ri["theta2"]) <= 1e-5


@pytest.mark.parametrize("sigma", [10.0, 20.0, 30.0, 50.0])
def test_denoise_512_sweep(dev, api, orc, sigma):
    # the 512x512 configuration (S = 10, K in {2, 3, 5}, beta = K/2) in the AVG order
    S = 10
    for K in (2, 3, 5):
        beta = K / 2.0
        img = synth.noisy_image(512, 512, sigma, seed=int(sigma) + K, dtype="f32")
        h = orc.default_h(sigma, K, "gauss_iir", beta)
        ref, _ = orc.snlm(img.astype(np.float64), S, K, h, "gauss_iir", beta, order="AVG")
        got = np_of(api.snlm_denoise(to_dev(img, dev), S, K, h, "gauss_iir", "AVG", 0.0, beta))
        assert np.abs(got - ref).max() <= TOL, (K, np.abs(got - ref).max())


@pytest.mark.parametrize("H,W,S,beta", [(97, 131, 10, 1.5), (1, 77, 5, 1.0), (64, 1, 6, 0.5), (1, 1, 3, 2.0),
                                         (5, 9, 20, 2.5), (3, 300, 7, 3.5), (41, 33, 0, 1.5), (600, 17, 30, 2.5)])
def test_denoise_shapes(dev, api, orc, H, W, S, beta):
    sigma = 25.0
    img = synth.noisy_image(H, W, sigma, seed=H * W + S, dtype="f32")
    h = orc.default_h(sigma, 3, "gauss_iir", beta)
    ref, _ = orc.snlm(img.astype(np.float64), S, 3, h, "gauss_iir", beta, order="RC")
    got = np_of(api.snlm_denoise(to_dev(img, dev), S, 3, h, "gauss_iir", "RC", 0.0, beta))
    assert np.abs(got - ref).max() <= TOL


def test_invariants(dev, api):
    import torch

    # constant image unchanged; h -> 0 is the identity
    c = torch.full((70, 90), 91.0, device=dev)
    out = np_of(api.snlm_denoise(c, 8, 3, 30.0, "gauss_iir", "AVG", 0.0, 1.5))
    assert np.abs(out - 91.0).max() <= 1e-4
    img = synth.noisy_image(80, 120, 20.0, seed=9, dtype="f32")
    out = np_of(api.snlm_denoise(to_dev(img, dev), 8, 3, 1e-20, "gauss_iir", "RC", 0.0, 1.5))
    np.testing.assert_array_equal(out, img)


def test_unsupported_and_invalid_requests(dev, api):
    import torch

    from paper_1407_2343_gb300 import _lib

    lib = _lib.load()
    img = torch.zeros((16, 16), dtype=torch.uint8, device=dev)
    out = torch.full((16, 16), 7.0, device=dev)
    p = lambda t: t.data_ptr()  # noqa: E731
    # beta outside [0.5, 3.5]
    assert lib.snlm_denoise(p(img), 0, 16, 16, 16, 5, 3, 10.0, 2, 0, 0.0, 0.4, p(out), None) == api.ERR_ARG
    assert lib.snlm_denoise(p(img), 0, 16, 16, 16, 5, 3, 10.0, 2, 0, 0.0, 3.6, p(out), None) == api.ERR_ARG
    assert lib.snlm_patch_dist_1d(p(img), 0, 16, 16, 16, 5, 3, 2, 4.0, p(out), None) == api.ERR_ARG
    # no derivative chain for this profile
    d = torch.zeros((16, 16), device=dev)
    assert lib.snlm_nlm_1d(p(img), 0, 16, 16, 16, 1, 5, 3, 10.0, 2, 1.5, p(out), 16, 1, None, p(d), None) == \
        api.ERR_UNSUPPORTED
    assert api.snlm_default_h(10.0, 3, "gauss_iir", 4.0) == -1.0
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
    # the batch plans do not run it
    with pytest.raises(api.SnlmError) as e:
        api.snlm_batch_plan_create([dict(img=img, out=out, S=5, K=3, h=10.0, profile="gauss_iir")])
    assert e.value.status == api.ERR_UNSUPPORTED


def test_other_entry_points_run_the_recursive_profile(dev, api, orc):
    # the host-buffer, pipelined, allocation-free and post-filtered entry points give
    # the device path's result (they share its passes), and the device path the oracle's
    import torch

    sigma, S, K, beta = 25.0, 8, 3, 1.5
    img = synth.noisy_image(120, 90, sigma, seed=12, dtype="u8")
    h = orc.default_h(sigma, K, "gauss_iir", beta)
    dev_out = np_of(api.snlm_denoise(to_dev(img, dev), S, K, h, "gauss_iir", "CR", 0.0, beta))
    ref, _ = orc.snlm(img.astype(np.float64), S, K, h, "gauss_iir", beta, order="CR")
    assert np.abs(dev_out - ref).max() <= TOL
    host = api.snlm_denoise_host(img, S, K, h, "gauss_iir", "CR", 0.0, beta)
    np.testing.assert_array_equal(np.asarray(host), dev_out)
    many = api.snlm_denoise_host_many([img, img], S, K, h, "gauss_iir", "CR", 0.0, beta)
    for o in many:
        np.testing.assert_array_equal(np.asarray(o), dev_out)
    out = torch.empty((120, 90), dtype=torch.float32, device=dev)
    api.snlm_denoise_noalloc(to_dev(img, dev), S, K, h, "gauss_iir", "CR", 0.0, beta, out=out)
    np.testing.assert_array_equal(np_of(out), dev_out)
    ss, sr = api.snlm_bf_params(sigma)
    bf = np_of(api.snlm_denoise_bf(to_dev(img, dev), S, K, h, "gauss_iir", "CR", sigma, beta))
    np.testing.assert_array_equal(bf, np_of(api.snlm_bilateral(to_dev(dev_out, dev), ss, sr)))


def test_trace_names_the_recursive_passes(dev, api):
    img = to_dev(synth.noisy_image(64, 64, 20.0, seed=1, dtype="u8"), dev)
    api.snlm_trace_enable(True)
    try:
        api.snlm_denoise(img, 5, 3, 40.0, "gauss_iir", "RC", 0.0, 1.5)
        names = [k for k, _ in api.snlm_trace_read()]
    finally:
        api.snlm_trace_enable(False)
    assert names[:2] == ["row_pass/iir", "col_pass/iir"]


def test_full_size_sampled_parity(dev, api, orc):
    # 4096x4096 uint8, S = 20, beta = 2.5 (K = 5), sigma = 30, AVG order: the launch
    # configuration the benchmark times for this profile. Sampled pixels of f_rc and
    # f_cr are compared with the oracle run on a crop whose borders lie farther from
    # the sample than two passes can reach: S plus the oracle's warm-up margin (beyond
    # which the filter's response is below 1e-30) per pass.
    H = W = 4096
    S, K, beta, sigma = 20, 5, 2.5, 30.0
    R = S + orc.iir_margin(beta)
    img = synth.noisy_image(H, W, sigma, seed=0, dtype="u8")
    t = to_dev(img, dev)
    h = orc.default_h(sigma, K, "gauss_iir", beta)
    rc = np_of(api.snlm_denoise(t, S, K, h, "gauss_iir", "RC", 0.0, beta))
    cr = np_of(api.snlm_denoise(t, S, K, h, "gauss_iir", "CR", 0.0, beta))
    avg = np_of(api.snlm_denoise(t, S, K, h, "gauss_iir", "AVG", 0.0, beta))
    assert np.abs(avg - 0.5 * (rc.astype(np.float64) + cr)).max() <= 1e-4
    rng = np.random.default_rng(1)
    pts = [(0, 0), (H - 1, W - 1), (5, 2500)] + [tuple(p) for p in rng.integers(0, 4096, size=(3, 2))]
    for (r, c) in pts:
        r0, c0 = max(0, r - 2 * R), max(0, c - 2 * R)
        r1, c1 = min(H, r + 2 * R + 1), min(W, c + 2 * R + 1)
        parts = orc.snlm_parts(img[r0:r1, c0:c1].astype(np.float64), S, K, h, "gauss_iir", beta)
        assert abs(rc[r, c] - parts["frc"][r - r0, c - c0]) <= TOL
        assert abs(cr[r, c] - parts["fcr"][r - r0, c - c0]) <= TOL
