"""The separable 3-D extension (1-D passes along x, y and z of a volume) on the GPU
against the FP64 oracle, within the 1e-4 tolerance of the 2-D passes (three passes
instead of two, each pass's error a few 1e-6 plus the float32 rounding of its
output)."""
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


def volume(D, H, W, dtype, seed):
    v = np.stack([synth.scene(H, W, 20.0, seed=seed + z).noisy for z in range(D)])
    return synth.store(v, dtype)


CASES = [
    # D, H, W, dtype, S, K, profile, order
    (5, 17, 23, "u8", 3, 2, "box", "XYZ"),
    (12, 12, 12, "f16", 4, 1, "gauss", "AVG6"),
    (3, 40, 9, "f32", 6, 3, "box", "AVG6"),
    (33, 8, 70, "u8", 10, 3, "box", "XYZ"),
    (2, 1, 1, "f32", 2, 1, "box", "AVG6"),
]


@pytest.mark.parametrize("D,H,W,dtype,S,K,prof,order", CASES)
def test_3d_matches_the_oracle(api, orc, D, H, W, dtype, S, K, prof, order):
    import torch

    vol = volume(D, H, W, dtype, seed=D * 100 + W)
    h = orc.default_h(20.0, K, prof)
    ref = orc.snlm_3d(vol.astype(np.float64), S, K, h, prof, order=order)
    got = api.snlm_denoise_3d(torch.from_numpy(vol).cuda(), S, K, h, prof, order3=order).cpu().numpy()
    assert np.abs(got - ref).max() <= TOL


def test_3d_with_one_slice_equals_the_rc_order_bitwise(api):
    import torch

    img = synth.noisy_image(70, 90, 20.0, seed=9, dtype="u8")
    t = torch.from_numpy(img).cuda()
    h = api.snlm_default_h(20.0, 3)
    rc = api.snlm_denoise(t, 8, 3, h, "box", "RC").cpu().numpy()
    v = api.snlm_denoise_3d(t[None].contiguous(), 8, 3, h, "box", order3="XYZ").cpu().numpy()[0]
    assert np.array_equal(v, rc)


def test_3d_at_a_video_size_on_a_block(api, orc):
    # 64 frames of 256 x 256, S = 10, K = 3. In the order XYZ a voxel depends on the
    # input within S + K along y and z (and on its whole row along x), so the oracle on
    # the block of the first 64 rows (all frames, whole rows; it starts at the image
    # edge, where its extension is the volume's) decides rows 0 .. 64 - (S + K) - 2.
    import torch

    D, H, W, S, K = 64, 256, 256, 10, 3
    vol = volume(D, H, W, "u8", seed=1)
    h = orc.default_h(20.0, K)
    got = api.snlm_denoise_3d(torch.from_numpy(vol).cuda(), S, K, h, order3="XYZ").cpu().numpy()
    ref = orc.snlm_3d(vol[:, :64, :].astype(np.float64), S, K, h, order="XYZ")
    keep = 64 - (S + K) - 1
    assert np.abs(got[:, :keep, :] - ref[:, :keep, :]).max() <= TOL


def test_3d_argument_errors(api):
    import ctypes

    import torch
    from paper_1407_2343_gb300 import _lib

    lib = _lib.load()
    v = torch.zeros((4, 8, 8), dtype=torch.uint8, device="cuda")
    out = torch.full((4, 8, 8), 7.0, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.snlm_denoise_3d(p(v), 0, 4, 8, 8, 3, 2, 10.0, 0, 0.0, 2, p(out), None) == api.ERR_ARG
    assert lib.snlm_denoise_3d(p(v), 0, 4, 8, 8, 3, 8, 10.0, 0, 0.0, 0, p(out), None) == api.ERR_UNSUPPORTED
    assert lib.snlm_denoise_3d(p(v), 0, 4, 8, 8, 3, 2, 0.0, 0, 0.0, 0, p(out), None) == api.ERR_ARG
    assert lib.snlm_denoise_3d(p(v), 0, 0, 8, 8, 3, 2, 10.0, 0, 0.0, 0, p(out), None) == api.ERR_ARG
    torch.cuda.synchronize()
    assert (out == 7.0).all()
