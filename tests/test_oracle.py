"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names what fixes the expected value: the paper's own PatchLift route
(Alg. 1, Eqs. (10), (13)), hand-worked tiny cases, library routines for special
cases (numpy/scipy symmetric filters), closed forms, finite differences of the
map for the divergence of Eq. (24), a numerical minimiser of the SURE objective
of Eq. (17), and values printed in the paper (tests/golden/paper_values.txt).
"""
import math
import os

import numpy as np
import pytest
from scipy import ndimage, optimize

import patchlift_ref as plr
from paper_1407_2343_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_values():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_values.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = [t.strip() for t in line.split("=", 1)]
            try:
                vals[k] = float(v)
            except ValueError:
                vals[k] = v.strip('"')
    return vals


# ---------------------------------------------------------------- boundary rule

@pytest.mark.parametrize("N", [1, 2, 3, 5, 8])
def test_ext_matches_numpy_symmetric_pad(orc, N):
    # numpy's 'symmetric' pad is the half-sample symmetric extension, repeated
    # for widths beyond the signal length.
    R = 3 * N + 4
    x = np.arange(N, dtype=np.float64)
    padded = np.pad(x, R, mode="symmetric")
    got = np.array([orc.ext_index(p, N) for p in range(-R, N + R)], dtype=np.float64)
    np.testing.assert_array_equal(got, padded)


def test_ext_closed_form(orc):
    for N in (1, 4, 7):
        assert orc.ext_index(-1, N) == 0
        assert orc.ext_index(N, N) == N - 1
        for x in range(-20, 20):
            assert orc.ext_index(x, N) == orc.ext_index(x + 2 * N, N)   # period 2N
            assert orc.ext_index(x, N) == orc.ext_index(-1 - x, N)      # mirror about -1/2


# ---------------------------------------------------------------- patch distances (Eq. (3))

def test_patch_dist_hand_worked_box(orc):
    # f = (0, 1, 3), S = K = 1, box. Extended: ... 1 0 | 0 1 3 | 3 1 ...
    # d(0,-1): (0,0,1) vs (1,0,0) -> 1+0+1 = 2;  d(0,+1): (0,0,1) vs (0,1,3) -> 0+1+4 = 5
    # d(1,-1): (0,1,3) vs (0,0,1) -> 5;          d(1,+1): (0,1,3) vs (1,3,3) -> 1+4+0 = 5
    # d(2,-1): (1,3,3) vs (0,1,3) -> 5;          d(2,+1): (1,3,3) vs (3,3,1) -> 4+0+4 = 8
    d = orc.patch_dist_1d(np.array([0.0, 1.0, 3.0]), S=1, K=1, prof="box")[0]
    expect = np.array([[2, 0, 5], [5, 0, 5], [5, 0, 8]], dtype=np.float64)
    np.testing.assert_array_equal(d, expect)


def test_patch_dist_hand_worked_gauss(orc):
    # f = (0, 2), S = 1, K = 1, beta = 1: g(+-1) = exp(-1/2), g(0) = 1.
    # Extended ... 2 0 | 0 2 | 2 0 ...;  patch(0) = (0,0,2), patch(1) = (0,2,2), patch(-1) = (2,0,0)
    # d(0,+1) = e*0 + 1*4 + e*0 = 4;  d(0,-1) = e*4 + 0 + e*4 = 8e
    # d(1,-1) = 4;  patch(2) = (2,2,0): d(1,+1) = e*4 + 0 + e*4 = 8e
    e = math.exp(-0.5)
    d = orc.patch_dist_1d(np.array([0.0, 2.0]), S=1, K=1, prof="gauss", beta=1.0)[0]
    expect = np.array([[8 * e, 0, 4], [4, 0, 8 * e]])
    np.testing.assert_allclose(d, expect, rtol=1e-15, atol=0)


@pytest.mark.parametrize("N,S,K,prof", [(16, 3, 2, "box"), (12, 5, 1, "gauss"), (9, 4, 4, "box"),
                                         (5, 6, 3, "gauss"), (3, 2, 3, "box"), (1, 2, 2, "box")])
def test_patch_dist_matches_paper_patchlift(orc, N, S, K, prof):
    # Second route: the paper's lifting pipeline on the symmetric extension.
    rng = np.random.default_rng(N * 100 + S * 10 + K)
    f = rng.integers(0, 256, size=N).astype(np.float64)
    beta = max(K / 2.0, 1e-3)
    d = orc.patch_dist_1d(f, S, K, prof, beta)[0]
    R = S + K
    fe = plr.extend(f, R)
    g = orc.profile(K, prof, beta)
    dl = plr.distances(fe, S, K, g)
    scale = (2 * K + 1) * 255.0 ** 2
    for i in range(N):
        for s in range(-S, S + 1):
            a = dl[(R + i + 1, R + i + s + 1)]
            assert abs(d[i, s + S] - a) <= 1e-12 * scale, (i, s, d[i, s + S], a)


@pytest.mark.parametrize("K,prof", [(0, "box"), (2, "box"), (3, "gauss"), (5, "box")])
def test_patch_dist_matches_library_filter(orc, K, prof):
    # Third route: d(i, s) is g-weighted correlation of the lifted difference
    # (f(x) - f(x+s))^2 along x; computed here with scipy.ndimage.correlate1d.
    N, S = 40, 6
    f = synth.signals(1, N, 20.0, seed=3, dtype="u8")[0].astype(np.float64)
    beta = max(K / 2.0, 1e-3)
    g = orc.profile(K, prof, beta)
    d = orc.patch_dist_1d(f, S, K, prof, beta)[0]
    R = S + K
    fe = plr.extend(f, R)
    for s in range(-S, S + 1):
        lifted = (fe - np.roll(fe, -s)) ** 2
        filt = ndimage.correlate1d(lifted, g, mode="constant")
        np.testing.assert_allclose(d[:, s + S], filt[R:R + N], rtol=1e-13, atol=1e-9)


def test_patch_dist_invariants(orc):
    rng = np.random.default_rng(11)
    for N, S, K in [(30, 5, 2), (7, 9, 3), (2, 3, 1)]:
        f = rng.integers(0, 256, size=N).astype(np.float64)
        d = orc.patch_dist_1d(f, S, K, "box")[0]
        assert np.all(d[:, S] == 0.0)                        # w_ii = 1
        assert np.all(d >= 0)
        assert np.all(d == np.round(d))                      # integer data, box: exact integers
        assert d.max() <= (2 * K + 1) * 255 ** 2
        for i in range(N):                                   # band symmetry d(i,s) = d(i+s,-s)
            for s in range(-S, S + 1):
                if 0 <= i + s < N:
                    assert d[i, s + S] == d[i + s, -s + S]
        # affine behaviour: shift-invariant, quadratic in scale
        d2 = orc.patch_dist_1d(3.0 * f + 17.0, S, K, "box")[0]
        np.testing.assert_allclose(d2, 9.0 * d, rtol=1e-14)


# ---------------------------------------------------------------- packed layout of Sec. II-B

def test_packing_index_and_length():
    # Eq. (10) against a direct count of Alg. 1's filling order, and the length formula.
    for n, S, K in [(10, 3, 2), (7, 0, 1), (12, 5, 0), (9, 8, 3)]:
        l = 0
        pos = {}
        for mu in range(1, S + 2):
            for nu in range(1, n - S - 1 + mu + 1):
                l += 1
                j = nu
                i = S + 1 - mu + nu
                pos[(i, j)] = l
            l += K
        for (i, j), p in pos.items():
            assert plr.packed_index(i, j, n, S, K) == p
        assert plr.packed_length(n, S, K) == pos[(n, n)]
        assert plr.packed_index(n, n, n, S, K) == plr.packed_length(n, S, K)
    assert plr.packed_length(10, 3, 2) == 40.0
    assert paper_values()["packing_length_formula"] == "(S+1)*(N-S/2)+K*S"


# ---------------------------------------------------------------- 1-D NLM (Eq. (4))

def test_nlm_constant_signal_unchanged(orc):
    for N, S, K in [(20, 5, 2), (3, 7, 4), (1, 2, 2)]:
        f = np.full(N, 123.25)
        fh = orc.nlm_1d(f, S, K, h=10.0)
        np.testing.assert_allclose(fh, f, rtol=0, atol=1e-12)


def test_nlm_h_to_zero_is_identity(orc):
    # w_ii = 1 and every other weight underflows; a tie d = 0 forces f(j) = f(i)
    # because the centre tap has g(0) = 1.
    f = synth.signals(3, 50, 25.0, seed=1, dtype="u8").astype(np.float64)
    for prof in ("box", "gauss"):
        fh = orc.nlm_1d(f, 6, 2, h=1e-30, prof=prof)
        np.testing.assert_array_equal(fh, f)


@pytest.mark.parametrize("N,S", [(40, 5), (6, 9), (1, 3), (17, 17)])
def test_nlm_h_to_infinity_is_window_mean(orc, N, S):
    # All weights -> 1: the mean of the 2S+1 extended window samples, which is
    # scipy's uniform filter in half-sample 'reflect' mode (repeated when S >= N).
    rng = np.random.default_rng(N + S)
    f = rng.uniform(0, 255, size=N)
    fh = orc.nlm_1d(f, S, 2, h=1e30)
    R = S + 2
    fe = plr.extend(f, R)
    expect = ndimage.uniform_filter1d(fe, 2 * S + 1, mode="constant")[R:R + N]
    np.testing.assert_allclose(fh, expect, rtol=1e-13, atol=1e-11)
    if S < N:
        np.testing.assert_allclose(fh, ndimage.uniform_filter1d(f, 2 * S + 1, mode="reflect"), rtol=1e-13, atol=1e-11)


def test_nlm_convex_combination(orc):
    f = synth.signals(4, 64, 30.0, seed=5, dtype="f32").astype(np.float64)
    S, K = 7, 3
    fh = orc.nlm_1d(f, S, K, h=orc.default_h(30.0, K))
    for row, out in zip(f, fh):
        fe = plr.extend(row, S)
        for i in range(len(row)):
            win = fe[i:i + 2 * S + 1]
            assert win.min() - 1e-9 <= out[i] <= win.max() + 1e-9


def test_nlm_reversal_and_affine_equivariance(orc):
    f = synth.signals(2, 45, 20.0, seed=9, dtype="f32").astype(np.float64)
    S, K, h = 6, 2, 40.0
    fh = orc.nlm_1d(f, S, K, h)
    np.testing.assert_allclose(orc.nlm_1d(f[:, ::-1], S, K, h), fh[:, ::-1], rtol=1e-13, atol=1e-10)
    np.testing.assert_allclose(orc.nlm_1d(-2.0 * f + 50.0, S, K, 2.0 * h), -2.0 * fh + 50.0, rtol=1e-13, atol=1e-9)


def test_nlm_matches_paper_patchlift_nlm(orc):
    # Alg. 2 with the lifted distances on the extended signal.
    for prof in ("box", "gauss"):
        f = synth.signals(1, 30, 20.0, seed=2, dtype="f32")[0].astype(np.float64)
        S, K = 4, 2
        beta = 1.0
        h = orc.default_h(20.0, K, prof, beta)
        fh = orc.nlm_1d(f, S, K, h, prof, beta)
        R = S + K
        fe = plr.extend(f, R)
        ref = plr.patchlift_nlm(fe, S, K, h, orc.profile(K, prof, beta), R, R + len(f))
        np.testing.assert_allclose(fh, ref, rtol=1e-11, atol=1e-9)


def test_fig2_exactness(orc):
    # Fig. 2: NLM and PatchLift-NLM agree to an MSE of order 1e-17 on a noisy 1-D
    # signal (sigma = 0.2, S = 10, K = 5, h = 1).
    pv = paper_values()
    S, K, h, sig = int(pv["fig2_S"]), int(pv["fig2_K"]), pv["fig2_h"], pv["fig2_sigma"]
    rng = np.random.default_rng(0)
    t = np.arange(128)
    clean = (t > 40).astype(float) - 0.5 * (t > 90) + 0.3 * np.sin(t / 9.0)
    f = clean + sig * rng.standard_normal(len(t))
    fh = orc.nlm_1d(f, S, K, h)
    R = S + K
    ref = plr.patchlift_nlm(plr.extend(f, R), S, K, h, orc.profile(K, "box"), R, R + len(f))
    mse = float(np.mean((fh - ref) ** 2))
    assert mse <= 100 * pv["fig2_mse_order"], mse


def test_two_d_nlm_with_line_patches_equals_row_pass(orc):
    # Eqs. (1)-(2) with a 1x(2K+1) patch and a 1x(2S+1) window (box), brute force.
    img = synth.noisy_image(6, 9, 20.0, seed=4, dtype="u8").astype(np.float64)
    S, K, h = 2, 1, 30.0
    H, W = img.shape
    R = S + K
    pad = np.pad(img, ((0, 0), (R, R)), mode="symmetric")
    out = np.empty_like(img)
    for r in range(H):
        for c in range(W):
            num = den = 0.0
            for dj in range(-S, S + 1):
                d = sum((pad[r, R + c + k] - pad[r, R + c + dj + k]) ** 2 for k in range(-K, K + 1))
                w = math.exp(-d / h ** 2)
                num += w * pad[r, R + c + dj]
                den += w
            out[r, c] = num / den
    parts = orc.snlm_parts(img, S, K, h)
    np.testing.assert_allclose(parts["fr"], out, rtol=1e-13, atol=1e-11)
    # the column pass of the transposed image is the same map
    np.testing.assert_allclose(orc.snlm_parts(img.T.copy(), S, K, h)["fc"], out.T, rtol=1e-13, atol=1e-11)


# ---------------------------------------------------------------- divergence (Eq. (24))

@pytest.mark.parametrize("prof,S,K", [("box", 5, 2), ("gauss", 6, 3), ("box", 3, 3), ("gauss", 2, 4)])
def test_divergence_matches_central_differences(orc, prof, S, K):
    f = synth.signals(1, 48, 20.0, seed=7, dtype="f32")[0].astype(np.float64)
    beta = max(K / 2.0, 1e-3)
    h = orc.default_h(20.0, K, prof, beta)
    _, dlt = orc.nlm_1d(f, S, K, h, prof, beta, with_delta=True)
    eps = 1e-3
    R = S + K
    for i in range(R, len(f) - R):
        fp = f.copy(); fp[i] += eps
        fm = f.copy(); fm[i] -= eps
        num = (orc.nlm_1d(fp, S, K, h, prof, beta)[i] - orc.nlm_1d(fm, S, K, h, prof, beta)[i]) / (2 * eps)
        assert abs(dlt[i] - num) <= 1e-6 * max(1.0, abs(num)), (i, dlt[i], num)


def test_divergence_chaining_matches_finite_differences_2d(orc):
    # Eqs. (21)-(22): delta_1 = d f_rc(i)/d f(i), delta_2 = d f_cr(i)/d f(i).
    img = synth.noisy_image(20, 22, 20.0, seed=8, dtype="f32").astype(np.float64)
    S, K = 3, 1
    h = orc.default_h(20.0, K)
    parts = orc.snlm_parts(img, S, K, h)
    eps = 1e-3
    for (r, c) in [(7, 8), (10, 12), (5, 15)]:
        p = img.copy(); p[r, c] += eps
        m = img.copy(); m[r, c] -= eps
        pp, mm = orc.snlm_parts(p, S, K, h), orc.snlm_parts(m, S, K, h)
        g1 = (pp["frc"][r, c] - mm["frc"][r, c]) / (2 * eps)
        g2 = (pp["fcr"][r, c] - mm["fcr"][r, c]) / (2 * eps)
        assert abs(parts["d1"][r, c] - g1) <= 1e-6 * max(1.0, abs(g1))
        assert abs(parts["d2"][r, c] - g2) <= 1e-6 * max(1.0, abs(g2))


# ---------------------------------------------------------------- Alg. 4 and SURE

def test_orders_are_consistent(orc):
    img = synth.noisy_image(24, 31, 20.0, seed=1, dtype="u8").astype(np.float64)
    S, K = 4, 2
    h = orc.default_h(20.0, K)
    rc, _ = orc.snlm(img, S, K, h, order="RC")
    cr, _ = orc.snlm(img, S, K, h, order="CR")
    avg, _ = orc.snlm(img, S, K, h, order="AVG")
    np.testing.assert_allclose(avg, 0.5 * (rc + cr), rtol=1e-14, atol=1e-12)
    # RC is the column map applied to the row map, built from the 1-D entry point
    fr = orc.nlm_1d(img, S, K, h)
    frc = orc.nlm_1d(fr.T.copy(), S, K, h).T
    np.testing.assert_allclose(rc, frc, rtol=1e-14, atol=1e-12)
    fc = orc.nlm_1d(img.T.copy(), S, K, h).T
    fcr = orc.nlm_1d(fc, S, K, h)
    np.testing.assert_allclose(cr, fcr, rtol=1e-14, atol=1e-12)


def _sure_phi(theta, f, frc, fcr, d1, d2, sigma):
    # Eq. (17) with Eqs. (14) and (18)
    ft = theta[0] * frc + theta[1] * fcr
    n = f.size
    return np.sum((ft - f) ** 2) / n - sigma ** 2 + 2 * sigma ** 2 / n * np.sum(theta[0] * d1 + theta[1] * d2)


@pytest.mark.parametrize("prof", ["box", "gauss"])
def test_sure_theta_minimises_phi(orc, prof):
    sigma = 25.0
    img = synth.noisy_image(40, 48, sigma, seed=3, dtype="f32").astype(np.float64)
    S, K = 5, 2
    beta = 1.0
    h = orc.default_h(sigma, K, prof, beta)
    out, info = orc.snlm(img, S, K, h, prof, beta, order="SURE", sigma=sigma)
    pr = orc.snlm_parts(img, S, K, h, prof, beta)
    args = (img, pr["frc"], pr["fcr"], pr["d1"], pr["d2"], sigma)
    res = optimize.minimize(_sure_phi, x0=np.array([0.5, 0.5]), args=args, method="BFGS",
                            options=dict(gtol=1e-12, maxiter=2000))
    th = np.array([info["theta1"], info["theta2"]])
    # compare objective values (the minimiser is flat along the ill-conditioned direction)
    assert _sure_phi(th, *args) <= res.fun + 1e-9 * abs(res.fun) + 1e-12
    np.testing.assert_allclose(out, th[0] * pr["frc"] + th[1] * pr["fcr"], rtol=1e-14, atol=1e-11)
    # the sums reported match the parts
    np.testing.assert_allclose(info["sum_d1"], pr["d1"].sum(), rtol=1e-12)
    np.testing.assert_allclose(info["A12"], np.sum(pr["frc"] * pr["fcr"]), rtol=1e-12)


def test_sure_tracks_true_mse(orc):
    # Stein's estimate (Eq. (17)) is unbiased for the MSE of Eq. (16); on a
    # 128x128 scene with known clean image it lands within a few percent.
    sigma = 20.0
    sc = synth.scene(128, 128, sigma, seed=0)
    f = sc.noisy
    S, K = 5, 2
    h = orc.default_h(sigma, K)
    pr = orc.snlm_parts(f, S, K, h)
    for th in ([1.0, 0.0], [0.0, 1.0], [0.5, 0.5], [0.8, 0.25]):
        th = np.array(th)
        phi = _sure_phi(th, f, pr["frc"], pr["fcr"], pr["d1"], pr["d2"], sigma)
        mse = np.mean((th[0] * pr["frc"] + th[1] * pr["fcr"] - sc.clean) ** 2)
        assert abs(phi - mse) <= 0.08 * mse, (th, phi, mse)


def test_sure_singular_system_uses_pseudo_inverse(orc):
    # Constant image: f_rc = f_cr = f exactly, A has rank one. The minimum-norm
    # solution splits the weight equally.
    img = np.full((12, 10), 80.0)
    sigma = 5.0
    out, info = orc.snlm(img, 3, 1, 20.0, order="SURE", sigma=sigma)
    assert info["theta1"] == pytest.approx(info["theta2"], rel=1e-12)
    # in the rank-one case theta1 + theta2 = (sum f^2 - sigma^2 (sum d1 + sum d2)/2) / sum f^2
    s2 = np.sum(img ** 2)
    expect = (s2 - sigma ** 2 * 0.5 * (info["sum_d1"] + info["sum_d2"])) / s2
    assert info["theta1"] + info["theta2"] == pytest.approx(expect, rel=1e-12)
    np.testing.assert_allclose(out, (info["theta1"] + info["theta2"]) * 80.0, rtol=1e-13)


def test_default_h_rule(orc):
    pv = paper_values()
    for K in range(0, 7):
        assert orc.default_h(1.0, K, "box") == pytest.approx(math.sqrt(2 * K + 1), rel=1e-15)
    # Gaussian at S=10, K=3 with the near-optimal beta = 2 falls in the paper's range
    hg = orc.default_h(1.0, 3, "gauss", pv["beta_near_optimal"])
    assert pv["h_over_sigma_gauss_min"] <= hg <= pv["h_over_sigma_gauss_max"]
    # box at K=3 sits at the top of the paper's range (sqrt(7) = 2.65)
    assert abs(orc.default_h(1.0, 3, "box") - pv["h_over_sigma_box_max"]) < 0.06


def test_oracle_rejects_bad_arguments(orc):
    with pytest.raises(ValueError):
        orc.nlm_1d(np.zeros(4), 2, 1, h=0.0)
    with pytest.raises(ValueError):
        orc.snlm(np.zeros((4, 4)), -1, 1, 1.0)


# ---- the bilateral post-filter of Sec. III-B (Eq. (BF)) and its parameter rules

def test_bf_parameter_rules_reproduce_the_printed_values(orc):
    # the cubic rules of Sec. IV-A against the values printed in the captions of the
    # two bilateral-filtering figures (sigma = 15 and 20) and in Sec. IV-A (sigma = 30),
    # at the precision the paper prints them
    pv = paper_values()
    ss, sr = orc.bf_params(15.0)
    assert round(ss, 2) == float(pv["bf_sigma_s_at_15"]) and round(sr) == float(pv["bf_sigma_r_at_15"])
    ss, sr = orc.bf_params(20.0)
    assert round(ss, 2) == float(pv["bf_sigma_s_at_20"]) and round(sr) == float(pv["bf_sigma_r_at_20"])
    _, sr = orc.bf_params(30.0)
    assert abs(sr - float(pv["bf_sigma_r_at_30"])) < 1.0


def _spatial_kernel(sigma_s):
    R = int(np.floor(3.0 * sigma_s))
    j = np.arange(-R, R + 1)
    w = np.exp(-(j[:, None] ** 2 + j[None, :] ** 2) / (2.0 * sigma_s ** 2))
    return w / w.sum()


@pytest.mark.parametrize("sigma_s", [0.4, 0.85, 1.0, 1.7])
def test_bilateral_with_flat_range_kernel_is_the_spatial_gaussian(orc, sigma_s):
    # sigma_r -> infinity leaves the normalised truncated spatial Gaussian on
    # [-3 sigma_s, 3 sigma_s]^2; scipy's 'reflect' mode is the half-sample
    # symmetric extension
    from scipy import ndimage

    img = np.random.default_rng(3).uniform(0, 255, (23, 31))
    got = orc.bilateral(img, sigma_s, 1e30)
    ref = ndimage.correlate(img, _spatial_kernel(sigma_s), mode="reflect")
    assert np.abs(got - ref).max() < 1e-9


def test_bilateral_with_sharp_range_kernel_is_the_identity(orc):
    img = np.random.default_rng(4).uniform(0, 255, (17, 19))
    assert np.abs(orc.bilateral(img, 1.2, 1e-30) - img).max() < 1e-12 * 255


def test_bilateral_constant_image_unchanged(orc):
    img = np.full((9, 13), 77.25)
    assert np.abs(orc.bilateral(img, 1.3, 20.0) - 77.25).max() < 1e-12


@pytest.mark.parametrize("x", [3, 4, 5, 6, 7, 8])
def test_bilateral_two_level_edge_closed_form(orc, x):
    # a vertical edge (a left of column c0, b from c0 on): the row offsets give the
    # same factor to both levels and cancel, leaving 1-D sums over the column offsets
    a, b, c0, sigma_s, sigma_r = 40.0, 140.0, 6, 1.1, 90.0
    img = np.full((15, 12), a)
    img[:, c0:] = b
    R = int(np.floor(3.0 * sigma_s))
    jx = np.arange(-R, R + 1)
    ws = np.exp(-jx ** 2 / (2.0 * sigma_s ** 2))
    same = (x - jx < c0) if x < c0 else (x - jx >= c0)
    g = np.exp(-(a - b) ** 2 / (2.0 * sigma_r ** 2))
    own, other = (a, b) if x < c0 else (b, a)
    expect = (own * ws[same].sum() + g * other * ws[~same].sum()) / (ws[same].sum() + g * ws[~same].sum())
    got = orc.bilateral(img, sigma_s, sigma_r)
    assert np.abs(got[4:11, x] - expect).max() < 1e-12


def test_bilateral_convex_and_symmetric(orc):
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 255, (21, 18))
    out = orc.bilateral(img, 0.9, 60.0)
    assert out.min() >= img.min() - 1e-9 and out.max() <= img.max() + 1e-9
    # symmetric support and extension: transposing or flipping commutes with the filter
    assert np.abs(orc.bilateral(img.T, 0.9, 60.0) - out.T).max() < 1e-12
    assert np.abs(orc.bilateral(img[::-1], 0.9, 60.0) - out[::-1]).max() < 1e-12
    assert np.abs(orc.bilateral(img[:, ::-1], 0.9, 60.0) - out[:, ::-1]).max() < 1e-12


def test_snlm_full_is_alg4_then_bilateral(orc):
    img = np.random.default_rng(6).uniform(0, 255, (24, 20))
    h = orc.default_h(20.0, 2)
    ft, _ = orc.snlm(img, 4, 2, h, order="SURE", sigma=20.0)
    ss, sr = orc.bf_params(20.0)
    assert np.array_equal(orc.snlm_full(img, 4, 2, h, order="SURE", sigma=20.0), orc.bilateral(ft, ss, sr))


# ---- the 2-D non-local means of Eqs. (1)-(2) (the comparison workload of Sec. IV-B)

@pytest.mark.parametrize("prof", ["box", "gauss"])
def test_nlm_2d_with_line_window_and_patch_is_the_1d_pass(orc, prof):
    # a 1 x (2S+1) window and a 1 x (2K+1) patch reduce Eqs. (1)-(2) to the row pass
    # of Eq. (4); the transposed shapes to the column pass
    img = synth.noisy_image(11, 14, 20.0, seed=8, dtype="u8").astype(np.float64)
    S, K, h = 3, 2, 35.0
    beta = 1.0
    fr = orc.snlm_parts(img, S, K, h, prof, beta)["fr"]
    fc = orc.snlm_parts(img, S, K, h, prof, beta)["fc"]
    np.testing.assert_allclose(orc.nlm_2d(img, (0, S), (0, K), h, prof, beta), fr, rtol=1e-13, atol=1e-11)
    np.testing.assert_allclose(orc.nlm_2d(img, (S, 0), (K, 0), h, prof, beta), fc, rtol=1e-13, atol=1e-11)


@pytest.mark.parametrize("S", [1, 3])
def test_nlm_2d_flat_weights_give_the_window_mean(orc, S):
    # h -> infinity: the mean of the (2S+1)^2 window, read through the symmetric
    # extension (scipy's 'reflect' mode)
    from scipy import ndimage

    img = np.random.default_rng(9).uniform(0, 255, (13, 17))
    got = orc.nlm_2d(img, S, 2, 1e30)
    ref = ndimage.uniform_filter(img, size=2 * S + 1, mode="reflect")
    assert np.abs(got - ref).max() < 1e-9


def test_nlm_2d_identity_constant_and_symmetry(orc):
    rng = np.random.default_rng(10)
    img = rng.uniform(0, 255, (12, 15))
    np.testing.assert_allclose(orc.nlm_2d(img, 2, 1, 1e-30), img, rtol=0, atol=1e-12)
    assert np.abs(orc.nlm_2d(np.full((9, 8), 33.5), 2, 2, 10.0) - 33.5).max() < 1e-12
    out = orc.nlm_2d(img, 2, 1, 60.0, "gauss", 1.0)
    np.testing.assert_allclose(orc.nlm_2d(img.T.copy(), 2, 1, 60.0, "gauss", 1.0), out.T, rtol=1e-13, atol=1e-11)
    assert out.min() >= img.min() - 1e-9 and out.max() <= img.max() + 1e-9


def test_nlm_2d_gaussian_patch_kernel_is_the_2d_gaussian(orc):
    # Eq. (2) written with the 2-D Gaussian exp(-|k|^2 / (2 alpha^2)) at one interior
    # pixel, against the oracle's product of 1-D profiles
    img = synth.noisy_image(12, 12, 20.0, seed=12, dtype="f32").astype(np.float64)
    S, K, h, alpha = 2, 2, 40.0, 1.3
    y, x = 6, 5
    num = den = 0.0
    for sy in range(-S, S + 1):
        for sx in range(-S, S + 1):
            d = 0.0
            for k1 in range(-K, K + 1):
                for k2 in range(-K, K + 1):
                    G = math.exp(-(k1 * k1 + k2 * k2) / (2 * alpha ** 2))
                    d += G * (img[y + k1, x + k2] - img[y + sy + k1, x + sx + k2]) ** 2
            w = math.exp(-d / h ** 2)
            num += w * img[y + sy, x + sx]
            den += w
    assert abs(orc.nlm_2d(img, S, K, h, "gauss", alpha)[y, x] - num / den) < 1e-10


# ---- the separable 3-D extension (Sec. V: separable NLM extends to volumes)

def test_3d_extension_with_one_slice_is_the_rc_order(orc):
    # along z a single slice is a signal of length 1, which every pass leaves as it is
    img = synth.noisy_image(14, 19, 20.0, seed=21, dtype="u8").astype(np.float64)
    S, K, h = 4, 2, 40.0
    ref, _ = orc.snlm(img, S, K, h, order="RC")
    got = orc.snlm_3d(img[None], S, K, h, order="XYZ")[0]
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-11)


def test_3d_extension_axis_labels(orc):
    # exchanging the x and z axes of the volume exchanges the roles of the passes
    vol = np.random.default_rng(22).uniform(0, 255, (5, 6, 7))
    S, K, h = 2, 1, 60.0
    a = orc.snlm_3d(vol, S, K, h, order="XYZ")
    b = orc.snlm_3d(np.ascontiguousarray(vol.transpose(2, 1, 0)), S, K, h, order="ZYX")
    np.testing.assert_allclose(b.transpose(2, 1, 0), a, rtol=1e-13, atol=1e-11)
    c = orc.snlm_3d(np.ascontiguousarray(vol.transpose(0, 2, 1)), S, K, h, order="YXZ")
    np.testing.assert_allclose(c.transpose(0, 2, 1), a, rtol=1e-13, atol=1e-11)


def test_3d_extension_constant_volume_and_average(orc):
    assert np.abs(orc.snlm_3d(np.full((3, 4, 5), 12.5), 2, 1, 10.0, order="AVG6") - 12.5).max() < 1e-12
    vol = np.random.default_rng(23).uniform(0, 255, (4, 5, 6))
    avg = orc.snlm_3d(vol, 2, 1, 50.0, order="AVG6")
    assert avg.min() >= vol.min() - 1e-9 and avg.max() <= vol.max() + 1e-9


# ---------------------------------------------------------------- closed form: a two-level step

def _step_nlm(N, c, a, b, S, K, h, g):
    # f = a left of c, b from c on; away from the ends the symmetric extension keeps
    # the step, and the patches centred at x and x+s differ exactly at the taps k
    # with x + k < c <= x + s + k (s > 0; mirrored for s < 0), each by (b - a)^2
    out = np.empty(N)
    for x in range(N):
        num = den = 0.0
        for s in range(-S, S + 1):
            lo, hi = (c - x - s, c - x - 1) if s > 0 else (c - x, c - x - s - 1)
            taps = [k for k in range(max(lo, -K), min(hi, K) + 1)]
            d2 = (b - a) ** 2 * sum(g[k + K] for k in taps) if s != 0 else 0.0
            w = math.exp(-d2 / (h * h))
            num += w * (a if x + s < c else b)
            den += w
        out[x] = num / den
    return out


@pytest.mark.parametrize("prof,K,beta", [("box", 3, None), ("gauss", 4, 1.5), ("box", 0, None)])
def test_nlm_of_a_step_matches_its_closed_form(orc, prof, K, beta):
    N, c, a, b, S, h = 60, 27, 10.0, 40.0, 6, 35.0
    x = np.where(np.arange(N) < c, a, b)
    g = orc.profile(K, prof, beta) if prof == "gauss" else np.ones(2 * K + 1)
    want = _step_nlm(N, c, a, b, S, K, h, g)
    got = orc.nlm_1d(x[None], S, K, h, prof, beta)[0]
    inner = slice(S + K, N - S - K)            # the extension keeps the step there
    np.testing.assert_allclose(got[inner], want[inner], rtol=1e-13, atol=1e-12)


def test_alg4_on_an_image_constant_along_columns_is_the_1d_closed_form(orc):
    # f(y, x) = step(x): every column is constant, so a column pass changes nothing
    # (all its patch distances are 0 and the window mean of equal samples is the
    # sample), and both orders of Alg. 4 reduce to the 1-D NLM of the step in each row
    N, c, a, b, S, K, h = 48, 21, 10.0, 40.0, 5, 2, 30.0
    row = np.where(np.arange(N) < c, a, b)
    img = np.tile(row, (17, 1))
    want = _step_nlm(N, c, a, b, S, K, h, np.ones(2 * K + 1))
    inner = slice(S + K, N - S - K)
    for order in ("RC", "CR", "AVG"):
        out, _ = orc.snlm(img, S, K, h, "box", order=order)
        np.testing.assert_allclose(out[:, inner], np.broadcast_to(want[inner], out[:, inner].shape),
                                   rtol=1e-13, atol=1e-12)
