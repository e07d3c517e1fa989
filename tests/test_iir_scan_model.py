"""The decomposition the CUDA recursive-profile pass uses, modelled in FP64 (CPU only).

The pass splits a line into tiles whose 512-position windows are spread over 32
lanes of 16 positions. Each recursion (causal, then anti-causal) runs over a lane's
run from rest to get the run's end state; a truncated Kogge-Stone scan over the
lanes, with powers of the 3x3 companion matrix, gives each lane its entering state;
the lane then runs again from it. Positions need `warm` samples of the window on both
sides, where `warm` is where the causal response has fallen below 1e-9 of its peak.
This model follows those steps in double precision with numpy and must reproduce the
oracle's sequential recursion, so a mistake in the decomposition (a wrong matrix
power, scan round, halo or mirrored offset) fails here without a GPU.
"""
import math

import numpy as np
import pytest

from paper_1407_2343_gb300 import synth

RUN, LANES = 16, 32
SPAN = RUN * LANES


def _plan(orc, beta):
    c = orc.iir_coeffs(beta)
    a = np.array([c["a1"], c["a2"], c["a3"]])
    A = np.array([[a[0], a[1], a[2]], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    w1 = w2 = w3 = 0.0
    peak, warm = 0.0, 0
    for n in range(4096):
        v = (c["B"] if n == 0 else 0.0) + a[0] * w1 + a[1] * w2 + a[2] * w3
        peak = max(peak, abs(v))
        if abs(v) > 1e-9 * peak:
            warm = n + 1
        w3, w2, w1 = w2, w1, v
    rounds = 0
    while (RUN << rounds) < warm:
        rounds += 1
    P = [np.linalg.matrix_power(A, RUN << d) for d in range(rounds)]
    return c, a, warm, rounds, P


def _runs(x, a, entering):
    """Recursion u(m) = x(m) + a1 u(m-1) + a2 u(m-2) + a3 u(m-3) over each lane's run
    (rows of x), from the given entering states (u(-1), u(-2), u(-3)) per lane."""
    out = np.empty_like(x)
    u1, u2, u3 = entering[:, 0].copy(), entering[:, 1].copy(), entering[:, 2].copy()
    for m in range(x.shape[1]):
        v = x[:, m] + a[0] * u1 + a[1] * u2 + a[2] * u3
        out[:, m] = v
        u3, u2, u1 = u2, u1, v
    return out


def _scan(ends, P, rounds):
    """Inclusive truncated Kogge-Stone scan S_r += P_d S_(r - 2^d); entering state of
    lane r is S_(r-1) (zero for lane 0)."""
    st = ends.copy()
    for d in range(rounds):
        sh = 1 << d
        shifted = np.zeros_like(st)
        shifted[sh:] = st[:-sh]
        st = st + shifted @ P[d].T
    enter = np.zeros_like(st)
    enter[1:] = st[:-1]
    return enter


def _filter_window(x, a, P, rounds):
    """Both passes over one window (x: LANES x RUN lifted squares), divided by B^2."""
    zero = np.zeros((LANES, 3))
    loc = _runs(x, a, zero)
    ends = np.stack([loc[:, -1], loc[:, -2], loc[:, -3]], 1)
    w = _runs(x, a, _scan(ends, P, rounds))
    # anti-causal: the same recursion on the reversed window (lanes and runs reversed)
    wr = w[::-1, ::-1]
    loc = _runs(wr, a, zero)
    ends = np.stack([loc[:, -1], loc[:, -2], loc[:, -3]], 1)
    y = _runs(wr, a, _scan(ends, P, rounds))
    return y[::-1, ::-1]


def model_dist(orc, f, S, beta):
    c, a, warm, rounds, P = _plan(orc, beta)
    N = len(f)
    T = SPAN - 2 * warm - S
    q0 = warm + S
    scale = beta * math.sqrt(2 * math.pi) * c["B"] ** 2
    ext = np.array([orc.ext_index(i, N) for i in range(-SPAN - 2 * S, N + SPAN + 2 * S)])
    off = SPAN + 2 * S
    out = np.full((N, 2 * S + 1), np.nan)
    out[:, S] = 0.0
    q = np.arange(SPAN)
    for t in range((N + T - 1) // T):
        b0 = t * T - q0
        fw = f[ext[off + b0 + np.arange(SPAN + S)]]
        for s in range(1, S + 1):
            dl = fw[q + s] - fw[q]
            y = _filter_window((dl * dl).reshape(LANES, RUN), a, P, rounds).ravel()
            d = scale * y
            x = b0 + q
            own = (q >= q0) & (q < q0 + T) & (x < N)
            out[x[own], S + s] = d[own]
            mir = (q + s >= q0) & (q + s < q0 + T) & (x + s < N)
            out[x[mir] + s, S - s] = d[mir]
    return out, warm, T


@pytest.mark.parametrize("N,S,beta", [(1500, 20, 2.5), (700, 5, 1.0), (1100, 40, 3.5), (9, 12, 0.5), (600, 0, 2.0)])
def test_scan_decomposition_reproduces_the_sequential_recursion(orc, N, S, beta):
    f = synth.signals(1, N, 30.0, seed=N + S, dtype="u8")[0].astype(np.float64)
    got, warm, T = model_dist(orc, f, S, beta)
    assert T > 0 and warm <= 64
    assert not np.isnan(got).any()
    ref = orc.patch_dist_1d(f[None], S, 0, "gauss_iir", beta)[0]
    # the model truncates the history where the response is below 1e-9 of its peak
    np.testing.assert_allclose(got, ref, rtol=1e-7, atol=1e-7 * ref.max())


def test_warm_up_lengths():
    # the history the pass needs at the widths the library takes (<= 64, two scan rounds)
    import oracle

    warms = {b: _plan(oracle, b)[2] for b in (0.5, 1.0, 2.5, 3.5)}
    assert warms == {0.5: 9, 1.0: 17, 2.5: 39, 3.5: 58}
