"""The host half of the banded SURE exchange: snlm_sure_theta (Eqs. (19), (25)
solved from seven sums in the basis m = (f_rc + f_cr)/2, d = (f_rc - f_cr)/2)
against the oracle's own solve of Alg. 4, on CPU (no device is touched)."""
import numpy as np
import pytest

from paper_1407_2343_gb300 import synth


def md_sums(f, frc, fcr, d1, d2):
    """The seven sums of a set of pixels in the m, d basis."""
    m, d = 0.5 * (frc + fcr), 0.5 * (frc - fcr)
    return [float((m * m).sum()), float((m * d).sum()), float((d * d).sum()), float((f * m).sum()),
            float((f * d).sum()), float(d1.sum()), float(d2.sum())]


@pytest.mark.parametrize("H,W,sigma,S,K", [(40, 52, 20.0, 5, 2), (33, 61, 35.0, 7, 3)])
def test_theta_from_sums_equals_the_oracle_solve(orc, H, W, sigma, S, K):
    from paper_1407_2343_gb300 import api

    f = synth.noisy_image(H, W, sigma, seed=H, dtype="f32").astype(np.float64)
    h = orc.default_h(sigma, K)
    p = orc.snlm_parts(f, S, K, h)
    _, info = orc.snlm(f, S, K, h, order="SURE", sigma=sigma)
    th = api.snlm_sure_theta(md_sums(f, p["frc"], p["fcr"], p["d1"], p["d2"]), sigma)
    assert th == pytest.approx((info["theta1"], info["theta2"]), rel=1e-9, abs=1e-12)
    # sums of disjoint row sets add: two halves give the same theta
    a = md_sums(f[:H // 2], p["frc"][:H // 2], p["fcr"][:H // 2], p["d1"][:H // 2], p["d2"][:H // 2])
    b = md_sums(f[H // 2:], p["frc"][H // 2:], p["fcr"][H // 2:], p["d1"][H // 2:], p["d2"][H // 2:])
    th2 = api.snlm_sure_theta(np.add(a, b), sigma)
    assert th2 == pytest.approx(th, rel=1e-12, abs=1e-14)


def test_theta_of_a_singular_system_is_the_minimum_norm_solution(orc):
    # a constant image: f_rc = f_cr, so d = 0 and the system is singular; theta is
    # the minimum-norm solution, theta1 = theta2 (the oracle's pseudo-inverse rule)
    from paper_1407_2343_gb300 import api

    f = np.full((24, 30), 100.0)
    sigma, S, K = 10.0, 4, 2
    h = orc.default_h(sigma, K)
    p = orc.snlm_parts(f, S, K, h)
    _, info = orc.snlm(f, S, K, h, order="SURE", sigma=sigma)
    th = api.snlm_sure_theta(md_sums(f, p["frc"], p["fcr"], p["d1"], p["d2"]), sigma)
    assert th[0] == pytest.approx(th[1], rel=1e-12)
    assert th == pytest.approx((info["theta1"], info["theta2"]), rel=1e-9)


def test_theta_rejects_bad_arguments():
    from paper_1407_2343_gb300 import api

    with pytest.raises(api.SnlmError):
        api.snlm_sure_theta([1.0, 0.0, 1.0, 1.0, 0.0, float("nan"), 0.0], 10.0)
    with pytest.raises(api.SnlmError):
        api.snlm_sure_theta([1.0, 0.0, 1.0, 1.0, 0.0, 0.0, 0.0], -1.0)
