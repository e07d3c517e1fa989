"""The persistent TMA passes against the FP64 oracle and against the gathering kernel.

With SNLM_OPT_TMA = 1, passes whose arrays allow bulk tensor copies (16-byte
aligned base, a stride that is a multiple of 16 bytes) run the TMA kernel; with 0
(the default) every pass runs the gathering kernel. Both must stay within the 1e-4 tolerance of the oracle, the
trace must show which kernel ran, and a wait that runs out (host-injected: the
barrier expects bytes that never arrive) must be reported without a device fault.
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
    yield api
    api.snlm_set_option(api.OPT_TMA, 0)
    api.snlm_set_option(api.OPT_INJECT_WAIT_TIMEOUT, 0)
    api.snlm_set_option(api.OPT_WAIT_LIMIT_US, 2000000)


def run(api, img, S, K, h, prof, order, sigma, beta, tma):
    import torch

    api.snlm_set_option(api.OPT_TMA, 1 if tma else 0)
    api.snlm_trace_read()
    api.snlm_trace_enable(True)
    try:
        out = api.snlm_denoise(torch.from_numpy(img).cuda(), S, K, h, prof, order, sigma, beta)
        torch.cuda.synchronize()
    finally:
        api.snlm_trace_enable(False)
        api.snlm_set_option(api.OPT_TMA, 0)
    names = [n for n, _ in api.snlm_trace_read()]
    assert api.snlm_device_error() == api.OK
    return out.cpu().numpy(), names


CASES = [
    # H, W, dtype, S, K, profile, order
    (256, 320, "u8", 20, 5, "box", "SURE"),
    (256, 320, "u8", 10, 3, "box", "RC"),
    (200, 256, "f16", 15, 2, "box", "CR"),
    (128, 192, "f32", 5, 5, "gauss", "AVG"),
    (64, 1024, "u8", 20, 5, "box", "SURE"),      # many tiles per row, few rows
    (1024, 48, "u8", 7, 1, "box", "SURE"),       # short rows: windows wider than the line
    (48, 64, "f32", 20, 7, "box", "SURE"),       # lines shorter than one window in both passes
    (96, 128, "u8", 0, 3, "box", "SURE"),        # S = 0: fhat = f
    (160, 160, "f32", 9, 0, "box", "RC"),        # K = 0
]


@pytest.mark.parametrize("H,W,dtype,S,K,prof,order", CASES)
def test_tma_and_gather_paths_match_the_oracle(api, orc, H, W, dtype, S, K, prof, order):
    sigma = 25.0
    beta = max(K / 2.0, 0.5)
    img = synth.noisy_image(H, W, sigma, seed=H + W + S, dtype=dtype)
    h = orc.default_h(sigma, K, prof, beta)
    ref, _ = orc.snlm(img.astype(np.float64), S, K, h, prof, beta, order=order, sigma=sigma)
    got_t, names_t = run(api, img, S, K, h, prof, order, sigma, beta, True)
    got_g, names_g = run(api, img, S, K, h, prof, order, sigma, beta, False)
    assert np.abs(got_t - ref).max() <= TOL
    assert np.abs(got_g - ref).max() <= TOL
    passes_t = [n for n in names_t if "pass" in n]
    assert passes_t and all(n.endswith("/tma") for n in passes_t), names_t
    assert not any(n.endswith("/tma") for n in names_g), names_g


def test_unaligned_layouts_fall_back_to_gathering(api, orc):
    # width 150 (8-bit rows of 150 bytes, float rows of 600 bytes): no tensor map
    sigma, S, K = 20.0, 8, 2
    img = synth.noisy_image(90, 150, sigma, seed=4, dtype="u8")
    h = orc.default_h(sigma, K)
    ref, _ = orc.snlm(img.astype(np.float64), S, K, h, "box", 1.0, order="SURE", sigma=sigma)
    got, names = run(api, img, S, K, h, "box", "SURE", sigma, 1.0, True)
    assert np.abs(got - ref).max() <= TOL
    assert names and not any(n.endswith("/tma") for n in names), names


def test_wait_timeout_is_reported_and_the_device_stays_usable(api, orc):
    import torch

    sigma, S, K = 20.0, 10, 3
    img = synth.noisy_image(256, 256, sigma, seed=7, dtype="u8")
    h = orc.default_h(sigma, K)
    t = torch.from_numpy(img).cuda()
    assert api.snlm_device_error() == api.OK
    api.snlm_set_option(api.OPT_TMA, 1)
    api.snlm_set_option(api.OPT_WAIT_LIMIT_US, 20000)
    api.snlm_set_option(api.OPT_INJECT_WAIT_TIMEOUT, 1)          # the first pass's waits run out
    try:
        out = api.snlm_denoise(t, S, K, h, "box", "RC", sigma)
        assert api.snlm_device_error() == api.ERR_TIMEOUT
        assert np.isnan(out.cpu().numpy()).all()
        assert api.snlm_get_option(api.OPT_INJECT_WAIT_TIMEOUT) == 0
    finally:
        api.snlm_set_option(api.OPT_INJECT_WAIT_TIMEOUT, 0)
        api.snlm_set_option(api.OPT_WAIT_LIMIT_US, 2000000)
        api.snlm_set_option(api.OPT_TMA, 0)
    assert api.snlm_device_error() == api.OK                      # the record was cleared
    ref, _ = orc.snlm(img.astype(np.float64), S, K, h, "box", 1.5, order="RC", sigma=sigma)
    out = api.snlm_denoise(t, S, K, h, "box", "RC", sigma)
    assert np.abs(out.cpu().numpy() - ref).max() <= TOL
    assert api.snlm_device_error() == api.OK


def test_options_are_validated(api):
    with pytest.raises(api.SnlmError):
        api.snlm_set_option(99, 1)
    with pytest.raises(api.SnlmError):
        api.snlm_set_option(api.OPT_WAIT_LIMIT_US, 0)
    with pytest.raises(api.SnlmError):
        api.snlm_set_option(api.OPT_TMA, 2)
    assert api.snlm_get_option(99) == -1
    assert api.snlm_get_option(api.OPT_TMA) == 0
