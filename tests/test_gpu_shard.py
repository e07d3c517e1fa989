"""Row bands of one image on one GPU: the banded result equals the unsharded one.

Each band is computed from its rows plus a halo of the column pass's reach (S + K,
or S + 64 for the recursive profile), and only its own rows are kept. Tile
boundaries inside a band differ from the whole image's, so float sums may round
differently: the comparison uses the float32 pixel tolerance, 1e-4 on [0, 255].
The SURE order adds the exchange of the seven sums (Eqs. (19), (25)): each band's
sums cover its own rows, their total gives the unsharded theta, and the bands'
sums are checked against the oracle's over the same rows.
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


@pytest.mark.parametrize("prof,S,K,beta", [("box", 10, 3, 0.0), ("gauss", 7, 5, 2.5), ("gauss_iir", 10, 5, 2.5)])
@pytest.mark.parametrize("order", ["RC", "CR", "AVG"])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_bands_equal_the_whole_image(dev, prof, S, K, beta, order, dtype):
    import torch

    from paper_1407_2343_gb300 import api, shard

    sigma = 25.0
    img = torch.from_numpy(synth.noisy_image(517, 300, sigma, seed=5, dtype=dtype)).to(dev)
    h = api.snlm_default_h(sigma, K, prof, beta)
    whole = api.snlm_denoise(img, S, K, h, prof, order, 0.0, beta)
    for n in (2, 3, 7):
        banded = shard.denoise_bands(img, S, K, h, prof, order, beta, n_bands=n)
        torch.cuda.synchronize()
        assert float((banded - whole).abs().max()) <= TOL, (n, float((banded - whole).abs().max()))


def test_bands_thinner_than_the_halo_and_the_oracle(dev, orc):
    import torch

    from paper_1407_2343_gb300 import api, shard

    sigma, S, K = 20.0, 6, 2
    img = synth.noisy_image(40, 33, sigma, seed=2, dtype="f32")
    h = orc.default_h(sigma, K)
    banded = shard.denoise_bands(torch.from_numpy(img).to(dev), S, K, h, "box", "AVG", n_bands=9)
    ref, _ = orc.snlm(img.astype(np.float64), S, K, h, "box", order="AVG")
    assert np.abs(banded.cpu().numpy() - ref).max() <= TOL
    with pytest.raises(ValueError):
        shard.denoise_bands(torch.from_numpy(img).to(dev), S, K, h, "box", "XY")


@pytest.mark.parametrize("prof,S,K,beta", [("box", 10, 3, 0.0), ("gauss", 7, 5, 2.5)])
@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_sure_bands_equal_the_whole_image_and_the_oracle(dev, orc, prof, S, K, beta, dtype):
    import torch

    from paper_1407_2343_gb300 import api, shard

    sigma = 25.0
    img_np = synth.noisy_image(517, 300, sigma, seed=5, dtype=dtype)
    img = torch.from_numpy(img_np).to(dev)
    h = api.snlm_default_h(sigma, K, prof, beta)
    info = torch.zeros(10, dtype=torch.float64, device=dev)
    whole = api.snlm_denoise_ws(img, S, K, h, prof, "SURE", sigma, beta, info=info)
    gi = info.cpu().numpy()
    ref, ri = orc.snlm(img_np.astype(np.float64), S, K, h, prof, beta, order="SURE", sigma=sigma)
    for n in (2, 3, 7):
        banded, theta = shard.denoise_bands(img, S, K, h, prof, "SURE", beta, n_bands=n, sigma=sigma)
        torch.cuda.synchronize()
        assert float((banded - whole).abs().max()) <= TOL, (n, float((banded - whole).abs().max()))
        assert abs(theta[0] - gi[0]) <= 1e-6 and abs(theta[1] - gi[1]) <= 1e-6, (n, theta, gi[:2])
        assert np.abs(banded.cpu().numpy() - ref).max() <= TOL
        assert abs(theta[0] - ri["theta1"]) <= 1e-6 and abs(theta[1] - ri["theta2"]) <= 1e-6


def test_sure_band_sums_cover_only_their_rows(dev, orc):
    # one band's seven sums against the oracle's over the same output rows
    import torch

    from paper_1407_2343_gb300 import api, shard

    sigma, S, K = 30.0, 8, 3
    img_np = synth.noisy_image(300, 257, sigma, seed=9, dtype="u8")
    f = img_np.astype(np.float64)
    h = orc.default_h(sigma, K)
    p = orc.snlm_parts(f, S, K, h)
    img = torch.from_numpy(img_np).to(dev)
    for band in shard.band_plan(300, 3, shard.reach(S, K)):
        r0, r1, h0, h1 = band
        _, _, sums = shard.sure_band(img, band, S, K, h)
        got = sums.cpu().numpy()
        sl = slice(r0, r1)
        m, d = 0.5 * (p["frc"][sl] + p["fcr"][sl]), 0.5 * (p["frc"][sl] - p["fcr"][sl])
        want = [(m * m).sum(), (m * d).sum(), (d * d).sum(), (f[sl] * m).sum(), (f[sl] * d).sum(),
                p["d1"][sl].sum(), p["d2"][sl].sum()]
        # sum m d and sum f d are sums of small differences of large terms: absolute bound
        for k, (g, w) in enumerate(zip(got, want)):
            assert abs(g - w) <= 1e-5 * abs(w) + 1e-4 * (r1 - r0) * 257, (band, k, g, w)


def test_sure_band_rejects_bad_rows(dev):
    import torch

    from paper_1407_2343_gb300 import api

    img = torch.zeros((40, 30), dtype=torch.uint8, device=dev)
    for r0, r1 in ((-1, 10), (10, 10), (5, 41)):
        with pytest.raises(api.SnlmError) as e:
            api.snlm_sure_band(img, 5, 2, 20.0, row0=r0, row1=r1)
        assert e.value.status == api.ERR_ARG
