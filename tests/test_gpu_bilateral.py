"""The bilateral post-filter of Sec. III-B (Eq. (BF)) and SNLM[f] on the GPU against
the FP64 oracle.

Tolerance. The kernel forms f(i) + sum_j wg_j t_j / sum_j wg_j (t_j = f(i-j) - f(i),
the centre weight 1). Each weight comes from one ex2.approx of an FP32 argument:
relative error <= ~2^-22 from the ex2 plus |arg| * 2^-24 * ln 2 from the rounded
argument (|arg| <= ~12 at the sizes here), so <= ~8e-7; the FP32 sums add <= ~(2R+1)^2
* 2^-24 relative. The error of the quotient is therefore below (8e-7 + 25 * 6e-8) *
max|t| = ~2.3e-6 * 255 ~= 6e-4 in the worst case (every large difference carrying a
large weight); on the synthetic scenes the observed error is ~1e-5. The tests hold
the filter alone to 2e-4 and SNLM[f] (whose input already carries the NLM passes'
~5e-5 error, damped by the filter's convex weights) to 2e-4.
"""
import numpy as np
import pytest

from paper_1407_2343_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 2e-4


@pytest.fixture(scope="module")
def api():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_2343_gb300 import _lib, api, build

    build.build()
    _lib.load()
    return api


def gpu_bf(api, x, ss, sr, pitch_pad=0):
    import torch

    H, W = x.shape
    buf = torch.zeros((H, W + pitch_pad), dtype=torch.float32, device="cuda")
    buf[:, :W] = torch.from_numpy(x.astype(np.float32))
    out = api.snlm_bilateral(buf[:, :W], ss, sr)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [
    # H, W, sigma_s, sigma_r, pitch padding
    (1, 1, 0.85, 144.0, 0),           # one pixel: every tap reflects onto it
    (3, 5, 2.9, 60.0, 3),             # R = 8 > the image: repeated reflection
    (37, 200, 0.85, 144.4, 0),        # the parameters of sigma = 30; ragged tile edges
    (130, 300, 0.7069, 77.1, 7),      # sigma = 15; padded pitch
    (64, 129, 1.0, 20.0, 0),          # R = 3; one column past a 16-byte boundary
    (50, 70, 0.3, 50.0, 0),           # R = 0: the identity
    (45, 61, 0.5, 1e6, 0),            # R = 1, flat range kernel
]


@pytest.mark.parametrize("H,W,ss,sr,pad", CASES)
def test_bilateral_matches_the_oracle(api, orc, H, W, ss, sr, pad):
    x = synth.noisy_image(H, W, 25.0, seed=H * 7 + W, dtype="f32").astype(np.float32)
    ref = orc.bilateral(x.astype(np.float64), float(np.float32(ss)), float(np.float32(sr)))
    got = gpu_bf(api, x, ss, sr, pad)
    assert np.abs(got - ref).max() <= TOL


def test_bilateral_identity_and_constant(api):
    x = synth.noisy_image(40, 90, 25.0, seed=1, dtype="f32").astype(np.float32)
    assert np.array_equal(gpu_bf(api, x, 0.3, 50.0), x)           # R = 0
    c = np.full((33, 47), 91.5, np.float32)
    assert np.array_equal(gpu_bf(api, c, 1.2, 30.0), c)           # every difference is 0


@pytest.mark.parametrize("order", ["SURE", "RC"])
def test_snlm_full_matches_the_oracle(api, orc, order):
    import torch

    sigma, S, K = 20.0, 10, 3
    img = synth.noisy_image(150, 210, sigma, seed=11, dtype="u8")
    h = orc.default_h(sigma, K)
    ss, sr = api.snlm_bf_params(sigma)
    assert abs(ss - orc.bf_params(sigma)[0]) < 1e-6 and abs(sr - orc.bf_params(sigma)[1]) < 1e-4
    ref = orc.snlm_full(img.astype(np.float64), S, K, h, order=order, sigma=sigma,
                        sigma_s=float(np.float32(ss)), sigma_r=float(np.float32(sr)))
    got = api.snlm_denoise_bf(torch.from_numpy(img).cuda(), S, K, h, "box", order, sigma)
    torch.cuda.synchronize()
    assert np.abs(got.cpu().numpy() - ref).max() <= TOL


def test_bilateral_at_full_size_on_sampled_rows(api, orc):
    # 4096^2 with the parameters of sigma = 30 (the benchmark's post-filter), rows
    # sampled across the image (the tile rows, the edges) against the oracle on the
    # rows with their R-row neighbourhood
    import torch

    n = 4096
    x = synth.noisy_image(n, n, 30.0, seed=2, dtype="f32").astype(np.float32)
    ss, sr = api.snlm_bf_params(30.0)
    R = int(np.floor(3.0 * np.float32(ss)))
    out = api.snlm_bilateral(torch.from_numpy(x).cuda(), ss, sr).cpu().numpy()
    for r in (0, 1, 15, 16, 2047, 2048, 4094, 4095):
        # the rows r - R .. r + R (reflected at the image edge) decide row r: a block
        # that holds them, and starts or ends at the image edge where they reflect,
        # gives the oracle the same extension
        lo, hi = max(0, r - R), min(n, r + R + 1)
        ref = orc.bilateral(x[lo:hi].astype(np.float64), float(np.float32(ss)), float(np.float32(sr)))
        assert np.abs(out[r] - ref[r - lo]).max() <= TOL, r


def test_bilateral_argument_errors(api):
    import ctypes

    import torch
    from paper_1407_2343_gb300 import _lib

    lib = _lib.load()
    x = torch.zeros((16, 16), device="cuda")
    out = torch.full((16, 16), 7.0, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.snlm_bilateral(p(x), 16, 16, 16, 0.0, 10.0, p(out), 16, None) == api.ERR_ARG
    assert lib.snlm_bilateral(p(x), 16, 16, 16, 1.0, -1.0, p(out), 16, None) == api.ERR_ARG
    assert lib.snlm_bilateral(p(x), 16, 16, 16, 3.0, 10.0, p(out), 16, None) == api.ERR_UNSUPPORTED   # R = 9
    assert lib.snlm_bilateral(p(x), 16, 16, 16, 1.0, 10.0, p(x), 16, None) == api.ERR_ARG             # in place
    assert lib.snlm_bilateral(p(x), 16, 16, 8, 1.0, 10.0, p(out), 16, None) == api.ERR_ARG             # pitch < W
    host = np.zeros((16, 16), np.float32)
    assert lib.snlm_bilateral(ctypes.c_void_p(host.ctypes.data), 16, 16, 16, 1.0, 10.0, p(out), 16,
                              None) == api.ERR_ARG
    torch.cuda.synchronize()
    assert (out == 7.0).all()
    with pytest.raises(api.SnlmError):
        api.snlm_bf_params(-1.0)


def test_bilateral_is_traced(api):
    import torch

    x = torch.rand((64, 64), device="cuda")
    api.snlm_trace_read()
    api.snlm_trace_enable(True)
    api.snlm_bilateral(x, 0.85, 100.0)
    torch.cuda.synchronize()
    api.snlm_trace_enable(False)
    names = [n for n, _ in api.snlm_trace_read()]
    assert names == ["bilateral"]
