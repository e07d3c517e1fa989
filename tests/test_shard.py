"""Host logic of the row-band split of one image (CPU only)."""
import pytest

from paper_1407_2343_gb300 import shard


@pytest.mark.parametrize("H,n,halo", [(1, 1, 0), (1, 4, 5), (7, 3, 2), (100, 4, 25), (4096, 8, 25), (33, 33, 40)])
def test_bands_cover_every_row_once_with_clipped_halos(H, n, halo):
    plan = shard.band_plan(H, n, halo)
    assert len(plan) == min(n, H)
    assert plan[0][0] == 0 and plan[-1][1] == H
    sizes = []
    for k, (r0, r1, h0, h1) in enumerate(plan):
        assert r0 < r1
        if k:
            assert r0 == plan[k - 1][1]            # contiguous, no overlap
        assert h0 == max(0, r0 - halo) and h1 == min(H, r1 + halo)
        sizes.append(r1 - r0)
    assert max(sizes) - min(sizes) <= 1


def test_reach_of_each_profile():
    assert shard.reach(20, 5, "box") == 25
    assert shard.reach(10, 3, "gauss") == 13
    assert shard.reach(20, 5, "gauss_iir") == 20 + shard.IIR_MAX_WARM


def test_rejections():
    with pytest.raises(ValueError):
        shard.band_plan(0, 2, 1)
    with pytest.raises(ValueError):
        shard.band_plan(10, 0, 1)
