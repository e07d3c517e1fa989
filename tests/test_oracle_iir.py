"""Pins of the oracle's recursive Gaussian profile (CPU only).

Sec. II-B computes the Gaussian distances of Eq. (3) in constant time per pair
with a recursive Gaussian filter (Young and van Vliet, 1995). The oracle runs that
filter in FP64 along each extended line; these tests fix it against things other
than its own recursion: the pole construction its published coefficients come
from, closed forms (unit DC gain, a linear ramp), the symmetry of the two-pass
response, a brute-force convolution with the impulse response, the poles' decay
behind the warm-up margin, the exact truncated Gaussian profile it approximates,
and the NLM invariants of Eq. (4).
"""
import math

import numpy as np
import pytest

from paper_1407_2343_gb300 import synth

BETAS = [0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5]


def _impulse(orc, beta, L=None):
    L = L or 4 * orc.iir_margin(beta)
    x = np.zeros(2 * L + 1)
    x[L] = 1.0
    return orc.iir_filter(x, beta), np.arange(-L, L + 1)


@pytest.mark.parametrize("beta", [0.5, 1.0, 2.0, 2.49, 2.5, 3.5, 8.0, 30.0])
def test_coefficients_follow_from_the_design_poles(orc, beta):
    # Young and van Vliet build the filter from the three poles m0, m1 +- i m2 of
    # their rational approximation of the Gaussian, scaled by q:
    #   b0 ~ (m0 + q)(m1^2 + m2^2 + 2 m1 q + q^2),
    #   b1 ~ q (2 m0 m1 + m1^2 + m2^2 + (2 m0 + 4 m1) q + 3 q^2),
    #   b2 ~ -q^2 (m0 + 2 m1 + 3 q),  b3 ~ q^3,
    # all divided by m0 (m1^2 + m2^2); their printed constants are these products,
    # rounded to about six digits.
    m0, m1, m2 = 1.16680, 1.10783, 1.40586
    c = orc.iir_coeffs(beta)
    q = c["q"]
    b0 = (m0 + q) * (m1 ** 2 + m2 ** 2 + 2 * m1 * q + q * q)
    b1 = q * (2 * m0 * m1 + m1 ** 2 + m2 ** 2 + (2 * m0 + 4 * m1) * q + 3 * q * q)
    b2 = -q * q * (m0 + 2 * m1 + 3 * q)
    b3 = q ** 3
    for key, want in (("a1", b1 / b0), ("a2", b2 / b0), ("a3", b3 / b0)):
        assert c[key] == pytest.approx(want, rel=2e-5), key
    # B = 1 - (a1 + a2 + a3) cancels, so the constants' rounding shows in absolute terms
    assert c["B"] == pytest.approx(1 - (b1 + b2 + b3) / b0, abs=2e-5)


def test_q_rule_branches(orc):
    # q grows with beta on each of the two published rules; they switch at
    # beta = 2.5 with a step of about 6 per cent (1.598 from the square-root rule,
    # 1.504 from the linear one), and q is linear in beta above 2.5
    for lo_b, hi_b in ((0.5, 2.5 - 1e-9), (2.5, 10.0)):
        qs = [orc.iir_coeffs(b)["q"] for b in np.linspace(lo_b, hi_b, 100)]
        assert np.all(np.diff(qs) > 0)
    lo, hi = orc.iir_coeffs(2.5 - 1e-9)["q"], orc.iir_coeffs(2.5)["q"]
    assert lo == pytest.approx(3.97156 - 4.14554 * math.sqrt(1 - 0.26891 * 2.5), rel=1e-8)
    assert 0.0 < lo - hi < 0.1
    assert orc.iir_coeffs(5.0)["q"] - orc.iir_coeffs(4.0)["q"] == pytest.approx(0.98711, rel=1e-9)


@pytest.mark.parametrize("beta", BETAS)
def test_unit_dc_gain_and_symmetric_response(orc, beta):
    h, k = _impulse(orc, beta)
    assert h.sum() == pytest.approx(1.0, abs=1e-12)
    # a causal pass followed by the same recursion run backwards is an even response
    np.testing.assert_allclose(h, h[::-1], rtol=0, atol=1e-15)
    # the peak sits at 0 and the response falls off on both sides
    assert np.argmax(h) == len(h) // 2
    assert h[len(h) // 2 + 1] < h[len(h) // 2]


@pytest.mark.parametrize("beta", BETAS)
def test_response_approximates_the_sampled_gaussian(orc, beta):
    # the published design approximates the Gaussian of standard deviation beta; the
    # approximation error of the 1995 rules is a few per cent of the peak, and their
    # response is slightly wider than beta (measured here: 8-24 per cent)
    h, k = _impulse(orc, beta)
    g = np.exp(-k * k / (2.0 * beta * beta))
    g /= g.sum()
    assert np.abs(h - g).max() <= 0.10 * g.max()
    sd = math.sqrt(float((h * k * k).sum()))
    assert beta * 1.0 <= sd <= beta * 1.25, sd


@pytest.mark.parametrize("beta", [0.5, 1.0, 2.5, 3.5, 10.0, 64.0])
def test_warm_up_margin_leaves_no_tail(orc, beta):
    # the margin claim of the oracle: the largest pole modulus raised to the margin
    # is below 1e-30 (poles from numpy, not from the oracle's recursion)
    c = orc.iir_coeffs(beta)
    rho = max(abs(np.roots([1.0, -c["a1"], -c["a2"], -c["a3"]])))
    assert rho < 1.0
    assert rho ** orc.iir_margin(beta) < 1e-30


def _brute_force_dist(orc, x, S, beta):
    # d^2(i, i+s) = beta sqrt(2 pi) * sum_k h(k) F(i+k, s) over the symmetric
    # extension (numpy's 'symmetric' pad), h the filter's impulse response
    h, k = _impulse(orc, beta)
    L = len(k) // 2
    N = len(x)
    fe = np.pad(x, L + S + 1, mode="symmetric")
    off = L + S + 1
    out = np.zeros((N, 2 * S + 1))
    for s in range(-S, S + 1):
        for i in range(N):
            a = fe[off + i + k] - fe[off + i + k + s]
            out[i, s + S] = beta * math.sqrt(2 * math.pi) * float((h * a * a).sum())
    return out


@pytest.mark.parametrize("N,S,beta", [(1, 2, 1.0), (5, 3, 2.0), (9, 9, 0.5), (16, 4, 3.5), (30, 6, 1.5)])
def test_distances_match_brute_force_convolution(orc, N, S, beta):
    x = synth.signals(1, N, 20.0, seed=N + S, dtype="f32")[0].astype(np.float64)
    got = orc.patch_dist_1d(x[None], S, 0, "gauss_iir", beta)[0]
    ref = _brute_force_dist(orc, x, S, beta)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-9)


@pytest.mark.parametrize("beta", [1.0, 2.5, 3.5])
def test_ramp_closed_form(orc, beta):
    # f(i) = a i gives F(i, s) = a^2 s^2 for every i away from the line's ends, so
    # the distance is beta sqrt(2 pi) a^2 s^2 there (unit DC gain)
    N, S, a = 1200, 7, 0.3
    x = a * np.arange(N, dtype=np.float64)
    d = orc.patch_dist_1d(x[None], S, 0, "gauss_iir", beta)[0]
    M = orc.iir_margin(beta) + S
    s = np.arange(-S, S + 1)
    want = beta * math.sqrt(2 * math.pi) * a * a * s * s
    np.testing.assert_allclose(d[M:N - M], np.broadcast_to(want, (N - 2 * M, 2 * S + 1)), rtol=1e-12, atol=1e-12)


def test_band_symmetry_and_zero_offset(orc):
    x = synth.signals(3, 90, 25.0, seed=5, dtype="u8").astype(np.float64)
    S = 6
    d = orc.patch_dist_1d(x, S, 0, "gauss_iir", 2.0)
    assert np.all(d[:, :, S] == 0.0)
    for s in range(1, S + 1):
        # d^2(i, i+s) = d^2(i+s, i) (Eq. (8))
        np.testing.assert_allclose(d[:, :-s, S + s], d[:, s:, S - s], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("beta", [1.0, 2.0, 3.0])
def test_close_to_the_exact_gaussian_profile(orc, beta):
    # the recursive profile approximates the (untruncated) Gaussian profile of
    # Eq. (3): with K = 8 beta the truncated sum is the Gaussian to 1e-13, and the
    # two distances differ by the filter's approximation error only
    x = synth.signals(2, 300, 25.0, seed=2, dtype="f32").astype(np.float64)
    S, K = 8, int(8 * beta)
    d_iir = orc.patch_dist_1d(x, S, 0, "gauss_iir", beta)
    d_fir = orc.patch_dist_1d(x, S, K, "gauss", beta)
    rel = np.abs(d_iir - d_fir).sum() / np.abs(d_fir).sum()
    assert rel < 0.15, rel


def test_default_h(orc):
    for beta in (0.5, 1.5, 3.5):
        assert orc.default_h(20.0, 3, "gauss_iir", beta) == pytest.approx(20.0 * math.sqrt(beta * math.sqrt(2 * math.pi)))


# ---------------------------------------------------------------- the 1-D NLM with the recursive profile

def test_nlm_invariants(orc):
    beta, S = 1.5, 5
    x = synth.signals(4, 120, 20.0, seed=8, dtype="f32").astype(np.float64)
    h = orc.default_h(20.0, 3, "gauss_iir", beta)
    # constant signal unchanged
    c = np.full((2, 50), 37.25)
    np.testing.assert_allclose(orc.nlm_1d(c, S, 3, h, "gauss_iir", beta), c, rtol=0, atol=1e-12)
    # convex combination of the extended window's samples
    y = orc.nlm_1d(x, S, 3, h, "gauss_iir", beta)
    for ln in range(x.shape[0]):
        fe = np.pad(x[ln], S, mode="symmetric")
        win = np.lib.stride_tricks.sliding_window_view(fe, 2 * S + 1)
        assert np.all(y[ln] >= win.min(1) - 1e-9) and np.all(y[ln] <= win.max(1) + 1e-9)
    # h -> 0: the identity (every other pair has a positive distance)
    np.testing.assert_allclose(orc.nlm_1d(x, S, 3, 1e-30, "gauss_iir", beta), x, rtol=0, atol=0)
    # h -> infinity: the mean of the 2S+1 extended window samples
    yinf = orc.nlm_1d(x, S, 3, 1e30, "gauss_iir", beta)
    for ln in range(x.shape[0]):
        fe = np.pad(x[ln], S, mode="symmetric")
        mean = np.lib.stride_tricks.sliding_window_view(fe, 2 * S + 1).mean(1)
        np.testing.assert_allclose(yinf[ln], mean, rtol=1e-12, atol=1e-10)


def test_nlm_uses_the_recursive_distances(orc):
    # Eq. (4) written out with the oracle's recursive distances
    beta, S, K = 2.5, 4, 5
    x = synth.signals(2, 40, 25.0, seed=1, dtype="u8").astype(np.float64)
    h = orc.default_h(25.0, K, "gauss_iir", beta)
    d = orc.patch_dist_1d(x, S, K, "gauss_iir", beta)
    y = orc.nlm_1d(x, S, K, h, "gauss_iir", beta)
    for ln in range(2):
        fe = np.pad(x[ln], S, mode="symmetric")
        win = np.lib.stride_tricks.sliding_window_view(fe, 2 * S + 1)
        w = np.exp(-d[ln] / (h * h))
        np.testing.assert_allclose(y[ln], (w * win).sum(1) / w.sum(1), rtol=1e-13)


def test_separable_orders(orc):
    beta, S, K, sigma = 1.5, 4, 3, 20.0
    img = synth.noisy_image(24, 31, sigma, seed=4, dtype="f32").astype(np.float64)
    h = orc.default_h(sigma, K, "gauss_iir", beta)
    parts = orc.snlm_parts(img, S, K, h, "gauss_iir", beta)
    rc, _ = orc.snlm(img, S, K, h, "gauss_iir", beta, order="RC")
    cr, _ = orc.snlm(img, S, K, h, "gauss_iir", beta, order="CR")
    avg, _ = orc.snlm(img, S, K, h, "gauss_iir", beta, order="AVG")
    np.testing.assert_array_equal(rc, parts["frc"])
    np.testing.assert_array_equal(cr, parts["fcr"])
    np.testing.assert_allclose(avg, 0.5 * (rc + cr), rtol=1e-15, atol=1e-12)
    # the row pass is the 1-D NLM of every row
    np.testing.assert_array_equal(parts["fr"], orc.nlm_1d(img, S, K, h, "gauss_iir", beta))
    np.testing.assert_array_equal(parts["fc"], orc.nlm_1d(img.T, S, K, h, "gauss_iir", beta).T)


def test_rejections(orc):
    x = np.zeros((1, 10))
    with pytest.raises(ValueError):
        orc.patch_dist_1d(x, 2, 0, "gauss_iir", 0.4)        # below the published range of the q rule
    with pytest.raises(ValueError):
        orc.nlm_1d(x, 2, 0, 1.0, "gauss_iir", 70.0)


# ---------------------------------------------------------------- divergence (Eq. (24)) and SURE

@pytest.mark.parametrize("S,beta", [(5, 1.5), (8, 2.5), (3, 0.5)])
def test_divergence_matches_central_differences(orc, S, beta):
    # Eq. (24) with the recursive profile: centre weight g(0) = beta sqrt(2 pi) h(0)
    # and the patch term over the whole window. Interior points only: near the ends
    # f(i) also enters the mirrored samples, which Eq. (24) leaves out.
    f = synth.signals(1, 220, 20.0, seed=7, dtype="f32")[0].astype(np.float64)
    h = orc.default_h(20.0, 3, "gauss_iir", beta)
    _, dlt = orc.nlm_1d(f, S, 3, h, "gauss_iir", beta, with_delta=True)
    eps = 1e-3
    for i in range(90, 130):
        fp = f.copy(); fp[i] += eps
        fm = f.copy(); fm[i] -= eps
        num = (orc.nlm_1d(fp, S, 3, h, "gauss_iir", beta)[i] - orc.nlm_1d(fm, S, 3, h, "gauss_iir", beta)[i]) / (2 * eps)
        assert abs(dlt[i] - num) <= 1e-6 * max(1.0, abs(num)), (i, dlt[i], num)


def test_sure_theta_minimises_phi(orc):
    from scipy import optimize

    sigma, S, beta = 25.0, 5, 1.5
    img = synth.noisy_image(40, 48, sigma, seed=3, dtype="f32").astype(np.float64)
    h = orc.default_h(sigma, 3, "gauss_iir", beta)
    out, info = orc.snlm(img, S, 3, h, "gauss_iir", beta, order="SURE", sigma=sigma)
    pr = orc.snlm_parts(img, S, 3, h, "gauss_iir", beta)

    def phi(theta):
        # Eq. (17) with Eqs. (14) and (18)
        ft = theta[0] * pr["frc"] + theta[1] * pr["fcr"]
        n = img.size
        return np.sum((ft - img) ** 2) / n - sigma ** 2 + 2 * sigma ** 2 / n * np.sum(theta[0] * pr["d1"] +
                                                                                      theta[1] * pr["d2"])

    res = optimize.minimize(phi, x0=np.array([0.5, 0.5]), method="BFGS", options=dict(gtol=1e-12, maxiter=2000))
    th = np.array([info["theta1"], info["theta2"]])
    assert phi(th) <= res.fun + 1e-9 * abs(res.fun) + 1e-12
    np.testing.assert_allclose(out, th[0] * pr["frc"] + th[1] * pr["fcr"], rtol=1e-14, atol=1e-11)


def test_nlm_of_a_step_matches_its_closed_form(orc):
    # a two-level step: the lifted squares of offset s are (b - a)^2 on the s samples
    # whose patch pairs straddle the step and zero elsewhere, so the distance is
    # beta sqrt(2 pi) (b - a)^2 times the impulse response summed over those taps
    beta, N, c, a, b, S, h = 2.0, 400, 190, 10.0, 40.0, 6, 60.0
    hr, k = _impulse(orc, beta)
    L = len(k) // 2
    x = np.where(np.arange(N) < c, a, b)
    got = orc.nlm_1d(x[None], S, 0, h, "gauss_iir", beta)[0]
    scale = beta * math.sqrt(2 * math.pi)
    for i in range(150, 230):                       # far from the line's ends
        num = den = 0.0
        for s in range(-S, S + 1):
            lo, hi = (c - i - s, c - i - 1) if s > 0 else (c - i, c - i - s - 1)
            d2 = scale * (b - a) ** 2 * sum(hr[L + kk] for kk in range(lo, hi + 1)) if s != 0 else 0.0
            w = math.exp(-d2 / (h * h))
            num += w * (a if i + s < c else b)
            den += w
        assert got[i] == pytest.approx(num / den, rel=1e-12, abs=1e-10)
