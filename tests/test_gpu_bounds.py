"""Global-memory write bounds of every kernel family, checked with canaries.

compute-sanitizer is not available on the GPU pool, so out-of-bounds writes are
looked for the other way round: each output (and the caller-provided workspace) is
a view into a larger buffer whose margins hold a sentinel pattern; after the call
the margins must be intact, and the outputs must still match the oracle. Shapes are
ragged (partial tiles in both directions, lines shorter than a window, a single
pixel) so that the tail branches of every kernel run.
"""
import numpy as np
import pytest

from paper_1407_2343_gb300 import synth

pytestmark = pytest.mark.gpu

GUARD = 4096              # floats (16 KiB) of margin on each side
SENTINEL = -12345.5


@pytest.fixture(scope="module")
def api():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_2343_gb300 import _lib, api, build

    build.build()
    _lib.load()
    return api


def guarded(n):
    """A float32 CUDA buffer of n elements with sentinel margins; returns (whole, inner)."""
    import torch

    whole = torch.full((n + 2 * GUARD,), SENTINEL, dtype=torch.float32, device="cuda")
    return whole, whole[GUARD:GUARD + n]


def margins_intact(whole):
    import torch

    torch.cuda.synchronize()
    return bool((whole[:GUARD] == SENTINEL).all() and (whole[-GUARD:] == SENTINEL).all())


SHAPES = [(1, 1), (37, 53), (130, 257), (9, 300), (260, 7)]


@pytest.mark.parametrize("H,W", SHAPES)
@pytest.mark.parametrize("order", ["SURE", "AVG", "CR"])
def test_denoise_output_and_workspace_stay_in_bounds(api, orc, H, W, order):
    import torch

    sigma, S, K = 20.0, 10, 3
    img = synth.noisy_image(H, W, sigma, seed=H * W, dtype="u8")
    h = orc.default_h(sigma, K)
    whole, out = guarded(H * W)
    nbytes = api.snlm_workspace_bytes(H, W, order)
    wsb = torch.full((nbytes + 2 * 1024,), 0xA5, dtype=torch.uint8, device="cuda")
    ws = wsb[1024:1024 + nbytes]
    api.snlm_denoise_ws(torch.from_numpy(img).cuda(), S, K, h, "box", order, sigma, out=out.view(H, W), workspace=ws)
    assert margins_intact(whole)
    assert bool((wsb[:1024] == 0xA5).all() and (wsb[-1024:] == 0xA5).all())
    ref, _ = orc.snlm(img.astype(np.float64), S, K, h, order=order, sigma=sigma)
    assert np.abs(out.view(H, W).cpu().numpy() - ref).max() <= 1e-4


@pytest.mark.parametrize("n,N,S,K", [(5, 3, 20, 5), (33, 129, 20, 5), (4, 700, 7, 2)])
def test_strided_pass_outputs_stay_in_bounds(api, orc, n, N, S, K):
    # fhat and delta_out as column blocks of wider row-major buffers
    import torch

    pitch = N + 5
    x = synth.signals(n, N, 20.0, seed=n + N, dtype="f32")
    h = orc.default_h(20.0, K)
    wf, bf = guarded(n * pitch)
    wd, bd = guarded(n * pitch)
    fhat = bf.view(n, pitch)[:, :N]
    dout = bd.view(n, pitch)[:, :N]
    api.snlm_nlm_1d(torch.from_numpy(x).cuda(), S, K, h, fhat=fhat, delta_out=dout)
    assert margins_intact(wf) and margins_intact(wd)
    pad_f = bf.view(n, pitch)[:, N:]
    assert bool((pad_f == SENTINEL).all()) and bool((bd.view(n, pitch)[:, N:] == SENTINEL).all())
    ref, _ = orc.nlm_1d(x.astype(np.float64), S, K, h, with_delta=True)
    assert np.abs(fhat.cpu().numpy() - ref).max() <= 1e-4


@pytest.mark.parametrize("n,N,S,K", [(3, 5, 20, 5), (40, 333, 12, 4)])
def test_patch_distances_stay_in_bounds(api, orc, n, N, S, K):
    import torch

    x = synth.signals(n, N, 20.0, seed=7, dtype="f32")
    whole, inner = guarded(n * N * (2 * S + 1))
    api.snlm_patch_dist_1d(torch.from_numpy(x).cuda(), S, K, out=inner.view(n, N, 2 * S + 1))
    assert margins_intact(whole)
    ref = orc.patch_dist_1d(x.astype(np.float64), S, K)
    got = inner.view(n, N, 2 * S + 1).cpu().numpy()
    assert np.allclose(got, ref, rtol=2e-6, atol=1e-3)


@pytest.mark.parametrize("H,W", SHAPES)
def test_post_filter_and_2d_nlm_stay_in_bounds(api, orc, H, W):
    import torch

    x = synth.noisy_image(H, W, 20.0, seed=3, dtype="f32").astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    pitch = W + 3
    whole, inner = guarded(H * pitch)
    out = inner.view(H, pitch)[:, :W]
    api.snlm_bilateral(xd, 1.0, 40.0, out=out)
    assert margins_intact(whole) and bool((inner.view(H, pitch)[:, W:] == SENTINEL).all())
    assert np.abs(out.cpu().numpy() - orc.bilateral(x.astype(np.float64), 1.0, 40.0)).max() <= 2e-4
    whole2, inner2 = guarded(H * W)
    h2 = orc.default_h_2d(20.0, 2)
    api.snlm_nlm_2d(xd, 3, 2, h2, out=inner2.view(H, W))
    assert margins_intact(whole2)
    assert np.abs(inner2.view(H, W).cpu().numpy() - orc.nlm_2d(x.astype(np.float64), 3, 2, h2)).max() <= 1e-4
