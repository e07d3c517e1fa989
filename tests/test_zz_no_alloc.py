"""snlm_denoise_noalloc: the entry point for callers that may not allocate device
memory at run time (its scratch is a fixed area compiled into the library).

Checked through the C ABI against snlm_denoise on two calls in a row (the second
call must not see the first call's leftovers in the shared scratch), within the
1e-4 max-abs tolerance used by the other parity tests; plus the rejection of an
image whose scratch would not fit. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1407_2343_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_2343_gb300 import _lib, build

    build.build()
    return _lib.load()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_denoise_twice(lib):
    import torch

    from paper_1407_2343_gb300 import api

    dev = torch.device("cuda:0")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(256, 256, "u8", 20.0, 10, 3, api.SURE), (300, 170, "f32", 30.0, 7, 2, api.AVG),
             (1024, 1024, "u8", 25.0, 20, 5, api.SURE)]
    for (H, W, dt, sigma, S, K, order) in cases:
        img = torch.from_numpy(synth.noisy_image(H, W, sigma, seed=H + W, dtype=dt)).to(dev)
        code = {"u8": api.U8, "f16": api.F16, "f32": api.F32}[dt]
        h = api.snlm_default_h(sigma, K)
        ref = torch.empty((H, W), dtype=torch.float32, device=dev)
        assert lib.snlm_denoise(_p(img), code, H, W, W, S, K, h, api.BOX, order, sigma, 0.0, _p(ref), s) == 0
        for _ in range(2):
            out = torch.full((H, W), -1.0, dtype=torch.float32, device=dev)
            rc = lib.snlm_denoise_noalloc(_p(img), code, H, W, W, S, K, h, api.BOX, order, sigma, 0.0,
                                          _p(out), s)
            assert rc == 0, api.snlm_status_str(rc)
            torch.cuda.synchronize()
            err = float((out - ref).abs().max())
            assert err <= TOL, (H, W, order, err)


def test_noalloc_rejects_images_beyond_its_scratch(lib):
    import torch

    from paper_1407_2343_gb300 import api

    dev = torch.device("cuda:0")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    H = W = 2048                                   # SURE needs ~48 MiB > 32 MiB
    assert api.snlm_workspace_bytes(H, W, "SURE") > api.NOALLOC_SCRATCH_BYTES
    img = torch.zeros((H, W), dtype=torch.uint8, device=dev)
    out = torch.full((H, W), 5.0, dtype=torch.float32, device=dev)
    rc = lib.snlm_denoise_noalloc(_p(img), api.U8, H, W, W, 10, 3, 30.0, api.BOX, api.SURE, 10.0, 0.0, _p(out), s)
    assert rc == api.ERR_ARG
    torch.cuda.synchronize()
    assert bool((out == 5.0).all())
