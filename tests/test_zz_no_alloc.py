"""snlm_denoise_noalloc: the entry point for callers that may not allocate device
memory at run time (real-time loops, plug-ins whose host owns all device memory,
fixed-footprint programs); its scratch is a fixed area compiled into the library.

Checked through the C ABI against snlm_denoise_ws with a caller workspace: both
run the same passes on the same inputs, so the results must be identical bit for
bit, on two calls in a row (the second call must not see the first call's
leftovers in the shared scratch). A fresh process checks the defining property:
once the library is loaded, calls at new geometries (fp16 storage, a row pitch
wider than the image) leave the device's free memory unchanged. Images whose
scratch would not fit are rejected before any work. This file is collected last
on purpose.
"""
import ctypes
import os
import subprocess
import sys

import pytest

from paper_1407_2343_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def _padded(img, pitch):
    """A device copy of `img` whose rows are `pitch` elements apart."""
    import torch

    H, W = img.shape
    buf = torch.zeros((H, pitch), dtype=img.dtype, device=img.device)
    buf[:, :W] = img
    return buf


CASES = [(256, 256, 256, "u8", 20.0, 10, 3, "SURE"), (300, 170, 176, "f32", 30.0, 7, 2, "AVG"),
         (1024, 1024, 1024, "u8", 25.0, 20, 5, "SURE"), (517, 389, 400, "f16", 40.0, 15, 5, "SURE"),
         (640, 480, 512, "f16", 15.0, 10, 3, "RC")]


@pytest.mark.gpu
def test_noalloc_equals_ws_bit_for_bit_twice(lib):
    import torch

    from paper_1407_2343_gb300 import api

    dev = torch.device("cuda:0")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for (H, W, pitch, dt, sigma, S, K, order) in CASES:
        img = _padded(torch.from_numpy(synth.noisy_image(H, W, sigma, seed=H + W, dtype=dt)).to(dev), pitch)
        code = {"u8": api.U8, "f16": api.F16, "f32": api.F32}[dt]
        ordc = {"RC": api.RC, "AVG": api.AVG, "SURE": api.SURE}[order]
        h = api.snlm_default_h(sigma, K)
        ref = torch.empty((H, W), dtype=torch.float32, device=dev)
        nws = api.snlm_workspace_bytes(H, W, order)
        ws = torch.empty(nws, dtype=torch.uint8, device=dev)
        assert lib.snlm_denoise_ws(_p(img), code, H, W, pitch, S, K, h, api.BOX, ordc, sigma, 0.0, _p(ref),
                                   _p(ws), ctypes.c_size_t(nws), None, s) == 0
        for _ in range(2):
            out = torch.full((H, W), -1.0, dtype=torch.float32, device=dev)
            rc = lib.snlm_denoise_noalloc(_p(img), code, H, W, pitch, S, K, h, api.BOX, ordc, sigma, 0.0,
                                          _p(out), s)
            assert rc == 0, api.snlm_status_str(rc)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (H, W, dt, order, float((out - ref).abs().max()))


# Run in a fresh process: every kernel is loaded eagerly and every buffer (inputs,
# outputs, the reference path's workspace) exists before the first reading of the
# device's free memory; after that only snlm_denoise_noalloc runs, at geometries it
# has not seen in this process.
_FRESH = r"""
import ctypes, sys
import torch
sys.path.insert(0, ROOT)
from paper_1407_2343_gb300 import _lib, api, synth
lib = _lib.load()
dev = torch.device("cuda:0")
s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
P = lambda t: ctypes.c_void_p(t.data_ptr())
# load the module with one small call
small = torch.from_numpy(synth.noisy_image(64, 64, 20.0, seed=1, dtype="u8")).to(dev)
o = torch.empty((64, 64), dtype=torch.float32, device=dev)
assert lib.snlm_denoise_noalloc(P(small), api.U8, 64, 64, 64, 5, 2, 30.0, api.BOX, api.RC, 20.0, 0.0, P(o), s) == 0
cases = [(1600, 1500, 1536, "f16", 30.0, 20, 5, api.SURE), (1201, 999, 1024, "f32", 20.0, 10, 3, api.AVG),
         (2048, 1900, 2000, "u8", 50.0, 15, 3, api.RC)]
bufs = []
for (H, W, pitch, dt, sigma, S, K, order) in cases:
    img = torch.zeros((H, pitch), dtype={"u8": torch.uint8, "f16": torch.float16, "f32": torch.float32}[dt],
                      device=dev)
    img[:, :W] = torch.from_numpy(synth.noisy_image(H, W, sigma, seed=H, dtype=dt)).to(dev)
    code = {"u8": api.U8, "f16": api.F16, "f32": api.F32}[dt]
    h = api.snlm_default_h(sigma, K)
    name = {api.RC: "RC", api.AVG: "AVG", api.SURE: "SURE"}[order]
    nws = api.snlm_workspace_bytes(H, W, name)
    ws = torch.empty(nws, dtype=torch.uint8, device=dev)
    ref = torch.empty((H, W), dtype=torch.float32, device=dev)
    out = torch.full((H, W), -1.0, dtype=torch.float32, device=dev)
    assert lib.snlm_denoise_ws(P(img), code, H, W, pitch, S, K, h, api.BOX, order, sigma, 0.0, P(ref), P(ws),
                               ctypes.c_size_t(nws), None, s) == 0
    bufs.append((img, code, H, W, pitch, S, K, h, order, sigma, ref, out))
torch.cuda.synchronize()
free0, _ = torch.cuda.mem_get_info()
for (img, code, H, W, pitch, S, K, h, order, sigma, ref, out) in bufs:
    for _ in range(2):
        rc = lib.snlm_denoise_noalloc(P(img), code, H, W, pitch, S, K, h, api.BOX, order, sigma, 0.0, P(out), s)
        assert rc == 0, api.snlm_status_str(rc)
torch.cuda.synchronize()
free1, _ = torch.cuda.mem_get_info()
for b in bufs:
    assert torch.equal(b[11], b[10]), (b[2], b[3])
assert free1 == free0, (free0, free1)
print("noalloc fresh-process check ok", free0)
"""


@pytest.mark.gpu
def test_noalloc_allocates_nothing_in_a_fresh_process(lib):
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    code = "ROOT = %r\n" % ROOT + _FRESH
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "fresh-process check ok" in r.stdout


@pytest.mark.gpu
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


def test_noalloc_documented_size_limits():
    """The largest square images the fixed scratch admits for every S, as the
    header states them: 1654 (SURE), 2047 (AVG), 2896 (RC, CR); one more row and
    column does not fit."""
    from paper_1407_2343_gb300 import api

    cap = api.NOALLOC_SCRATCH_BYTES
    for order, n in (("SURE", 1654), ("AVG", 2047), ("RC", 2896), ("CR", 2896)):
        assert api.snlm_workspace_bytes(n, n, order) <= cap, order
        assert api.snlm_workspace_bytes(n + 1, n + 1, order) > cap, order
