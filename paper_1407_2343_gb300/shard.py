"""Row bands of one image (the split a multi-GPU run of a single large image would use).

Alg. 4 with the RC, CR or AVG order needs no exchange between bands of rows: a row
pass reads only its own row, and a column pass at row y reads the rows within its
reach (S + K for the exact profiles of Eq. (3); S plus the recursive filter's
history, at most 64 samples, for the recursive Gaussian). So a band of output rows
[r0, r1) is computed exactly from the input rows [r0 - reach, r1 + reach) clipped to
the image. A band's own edges are extended differently from the image's, and that
difference stays within the halo. The SURE order would add one exchange: an
all-reduce of the seven sums of Eqs. (19) and (25) before the combination. The
library's sums cover a whole call, halo rows included, so SURE is not split here.

`band_plan` is host logic only; `denoise_bands` runs each band through
`snlm_denoise` on a pitched view of the image and keeps its interior rows. Both
serve tests on one GPU, where the banded result must equal the unsharded one.
"""
from __future__ import annotations

from . import api

# Largest history of the recursive profile's passes (samples); beyond it the causal
# response of the filter is below 1e-9 of its peak for every width the library takes.
IIR_MAX_WARM = 64


def reach(S: int, K: int, profile="box") -> int:
    """Rows a column pass at row y reads on each side of y."""
    return S + (IIR_MAX_WARM if api._profile(profile) == api.GAUSS_IIR else K)


def band_plan(H: int, n_bands: int, halo: int):
    """Split rows [0, H) into n_bands bands of nearly equal size. Returns a list of
    (r0, r1, h0, h1): output rows [r0, r1), input rows [h0, h1) = the band widened by
    `halo` on each side and clipped to the image."""
    if H < 1 or n_bands < 1 or halo < 0:
        raise ValueError("need H >= 1, n_bands >= 1, halo >= 0")
    n = min(n_bands, H)
    plan = []
    for b in range(n):
        r0, r1 = b * H // n, (b + 1) * H // n
        plan.append((r0, r1, max(0, r0 - halo), min(H, r1 + halo)))
    return plan


def denoise_bands(img, S: int, K: int, h: float, profile="box", order="RC", beta: float = 0.0,
                  n_bands: int = 2, out=None, stream=None):
    """Alg. 4 (RC, CR or AVG) of a 2-D device tensor, band by band. Returns the
    H x W float32 result."""
    torch = api._torch()
    if str(order).upper() not in ("RC", "CR", "AVG"):
        raise ValueError("the banded split covers the RC, CR and AVG orders")
    H, W = img.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    for r0, r1, h0, h1 in band_plan(H, n_bands, reach(S, K, profile)):
        part = api.snlm_denoise(img[h0:h1], S, K, h, profile, order, 0.0, beta, stream=stream)
        out[r0:r1].copy_(part[r0 - h0:r1 - h0])
    return out
