"""Row bands of one image (the split a multi-GPU run of a single large image would use).

Alg. 4 with the RC, CR or AVG order needs no exchange between bands of rows: a row
pass reads only its own row, and a column pass at row y reads the rows within its
reach (S + K for the exact profiles of Eq. (3); S plus the recursive filter's
history, at most 64 samples, for the recursive Gaussian). So a band of output rows
[r0, r1) is computed exactly from the input rows [r0 - reach, r1 + reach) clipped to
the image. A band's own edges are extended differently from the image's, and that
difference stays within the halo. The SURE order adds one exchange: the seven sums
of Eqs. (19) and (25) (with the divergences of Eq. (24)) are sums over pixels, so
each band forms them over its own output rows (`snlm_sure_band`), the bands' sums
are added (an all-reduce across ranks), and every band solves the same 2x2 system
(`snlm_sure_theta`) and combines its own rows (`snlm_sure_combine`).

`band_plan` is host logic only; `denoise_bands` runs each band through the library
on a pitched view of the image and keeps its interior rows; `sure_band` and
`sure_finish_band` are the two halves of a SURE band around the exchange. They serve
tests on one GPU, where the banded result must equal the unsharded one, and the
two-rank test, where the exchange is a gloo all-reduce.
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


def sure_band(img, band, S: int, K: int, h: float, profile="box", beta: float = 0.0, stream=None):
    """The part of a SURE band before the exchange: f_rc and f_cr of the band's input
    rows and the seven sums over its output rows. `band` is one (r0, r1, h0, h1) of
    band_plan. Returns (f_rc, f_cr, sums) on the device."""
    r0, r1, h0, h1 = band
    return api.snlm_sure_band(img[h0:h1], S, K, h, profile, beta, r0 - h0, r1 - h0, stream=stream)


def sure_finish_band(band, f_rc, f_cr, theta, out, stream=None):
    """The part after the exchange: out[r0:r1] = theta1 f_rc + theta2 f_cr on the
    band's output rows."""
    r0, r1, h0, _ = band
    api.snlm_sure_combine(f_rc[r0 - h0:r1 - h0], f_cr[r0 - h0:r1 - h0], theta, out=out[r0:r1], stream=stream)


def denoise_bands(img, S: int, K: int, h: float, profile="box", order="RC", beta: float = 0.0,
                  n_bands: int = 2, out=None, stream=None, sigma: float = 0.0):
    """Alg. 4 of a 2-D device tensor, band by band. RC, CR and AVG need no exchange;
    SURE adds the sums of the bands (here on the host) before the combination.
    Returns the H x W float32 result (and, for SURE, theta as a second value)."""
    import numpy as np

    torch = api._torch()
    order = str(order).upper()
    if order not in ("RC", "CR", "AVG", "SURE"):
        raise ValueError("order must be RC, CR, AVG or SURE")
    H, W = img.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    plan = band_plan(H, n_bands, reach(S, K, profile))
    if order != "SURE":
        for r0, r1, h0, h1 in plan:
            part = api.snlm_denoise(img[h0:h1], S, K, h, profile, order, 0.0, beta, stream=stream)
            out[r0:r1].copy_(part[r0 - h0:r1 - h0])
        return out
    parts = [sure_band(img, b, S, K, h, profile, beta, stream) for b in plan]
    total = np.zeros(7)
    for _, _, sums in parts:
        total += sums.cpu().numpy()
    theta = api.snlm_sure_theta(total, sigma)
    for b, (f_rc, f_cr, _) in zip(plan, parts):
        sure_finish_band(b, f_rc, f_cr, theta, out, stream)
    return out, theta
