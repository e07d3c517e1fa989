"""Row bands of one image on one GPU: the banded result equals the unsharded one.

Each band is computed from its rows plus a halo of the column pass's reach (S + K,
or S + 64 for the recursive profile), and only its own rows are kept. Tile
boundaries inside a band differ from the whole image's, so float sums may round
differently: the comparison uses the float32 pixel tolerance, 1e-4 on [0, 255].
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
        shard.denoise_bands(torch.from_numpy(img).to(dev), S, K, h, "box", "SURE")
