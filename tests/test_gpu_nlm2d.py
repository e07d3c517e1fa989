"""The 2-D non-local means of Eqs. (1)-(2) on the GPU against the FP64 oracle.

Tolerance 1e-4 on the [0, 255] scale, as for the 1-D passes: the GPU forms the
patch distance as two FP32 1-D filters of the squared differences (exact integers
for uint8 with the box profile), one ex2 per offset, and the result in centred form
f(i) + sum w (f(j) - f(i)) / sum w (the offset 0 weighs 1), so the error is a few
ulp of the weights times the differences that carry weight.
"""
import numpy as np
import pytest

from paper_1407_2343_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def api():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_2343_gb300 import _lib, api, build

    build.build()
    _lib.load()
    return api


CASES = [
    # H, W, dtype, S, K, profile
    (40, 50, "f32", 3, 2, "box"),
    (33, 70, "u8", 5, 3, "gauss"),
    (24, 31, "u8", 20, 5, "box"),          # window and patch wider than the image: repeated reflection
    (1, 1, "f32", 2, 1, "box"),
    (45, 37, "f16", 4, 0, "box"),          # K = 0: pixel-wise weights
    (30, 41, "f32", 0, 3, "gauss"),        # S = 0: the identity
    (64, 96, "u8", 7, 7, "gauss"),         # the largest patch
]


@pytest.mark.parametrize("H,W,dtype,S,K,prof", CASES)
def test_nlm_2d_matches_the_oracle(api, orc, H, W, dtype, S, K, prof):
    import torch

    sigma = 20.0
    img = synth.noisy_image(H, W, sigma, seed=H + 3 * W, dtype=dtype)
    h = orc.default_h_2d(sigma, K, prof)
    ref = orc.nlm_2d(img.astype(np.float64), S, K, h, prof)
    got = api.snlm_nlm_2d(torch.from_numpy(img).cuda(), S, K, h, prof).cpu().numpy()
    assert np.abs(got - ref).max() <= TOL


def test_nlm_2d_comparison_size_on_sampled_pixels(api, orc):
    # 256^2, S = 20, K = 5, box (the paper's run-time table): every pixel of rows
    # sampled across the image against the oracle on crops holding each row's
    # (S+K)-neighbourhood (a crop that reaches the image edge starts or ends there,
    # so its extension is the image's)
    import torch

    n, S, K, sigma = 256, 20, 5, 30.0
    img = synth.noisy_image(n, n, sigma, seed=5, dtype="u8")
    h = orc.default_h_2d(sigma, K)
    got = api.snlm_nlm_2d(torch.from_numpy(img).cuda(), S, K, h).cpu().numpy()
    R = S + K
    for r in (0, 13, 128, 255):
        lo, hi = max(0, r - R), min(n, r + R + 1)
        ref = orc.nlm_2d(img[lo:hi].astype(np.float64), S, K, h)
        assert np.abs(got[r] - ref[r - lo]).max() <= TOL, r


def test_nlm_2d_argument_errors(api):
    import ctypes

    import torch
    from paper_1407_2343_gb300 import _lib

    lib = _lib.load()
    x = torch.zeros((16, 16), dtype=torch.uint8, device="cuda")
    out = torch.full((16, 16), 7.0, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.snlm_nlm_2d(p(x), 0, 16, 16, 16, 33, 2, 10.0, 0, 0.0, p(out), None) == api.ERR_UNSUPPORTED
    assert lib.snlm_nlm_2d(p(x), 0, 16, 16, 16, 3, 8, 10.0, 0, 0.0, p(out), None) == api.ERR_UNSUPPORTED
    assert lib.snlm_nlm_2d(p(x), 0, 16, 16, 16, 3, 2, 0.0, 0, 0.0, p(out), None) == api.ERR_ARG
    assert lib.snlm_nlm_2d(p(x), 0, 16, 16, 8, 3, 2, 10.0, 0, 0.0, p(out), None) == api.ERR_ARG
    assert lib.snlm_nlm_2d(p(x), 9, 16, 16, 16, 3, 2, 10.0, 0, 0.0, p(out), None) == api.ERR_ARG
    torch.cuda.synchronize()
    assert (out == 7.0).all()
