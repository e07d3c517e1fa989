"""The paper's own PatchLift pipeline, written for the tests as a second,
independent route to the patch distances (Sec. II-A/B, Alg. 1, Eqs. (10), (13)).

It lifts a signal into the tensor product F(i,j) = f(i) f(j) (Eq. (5)), packs the
sub-diagonals of the band B (Eq. (8)) into one sequence V with K zeros between
them (Alg. 1), filters V with g_beta (Eq. (11)), and reads distances back with the
closed-form index l_ij of Eq. (10) and the three-sample rule of Eq. (13).

It is used only to pin the oracle, which computes Eq. (3) directly.
Indices here are 1-based, as in the paper.
"""
from __future__ import annotations

import numpy as np


def packed_index(i: int, j: int, n: int, S: int, K: int) -> int:
    """Eq. (10): position of F(i, j), i >= j, i - j <= S, in the packed sequence."""
    return ((S - i + j) * (2 * n + 2 * K - S - 1 - i + j)) // 2 + j


def packed_length(n: int, S: int, K: int) -> float:
    """Sec. II-B: L = (S+1)(n - S/2) + K S."""
    return (S + 1) * (n - S / 2.0) + K * S


def build_V(f: np.ndarray, S: int, K: int) -> np.ndarray:
    """Alg. 1, first part: V[l] (1-based; V[0] unused) for the signal f."""
    n = len(f)
    L = int(round(packed_length(n, S, K)))
    V = np.zeros(L + 1)
    l = 0
    for mu in range(1, S + 2):
        for nu in range(1, n - S - 1 + mu + 1):
            l += 1
            V[l] = f[S + 1 - mu + nu - 1] * f[nu - 1]
        l += K
    return V


def filtered_V(f: np.ndarray, S: int, K: int, g: np.ndarray) -> np.ndarray:
    """Alg. 1: Vbar = V * g_beta (g symmetric, support [-K, K])."""
    V = build_V(f, S, K)
    body = np.convolve(V[1:], g[::-1], mode="full")[K:K + len(V) - 1]
    return np.concatenate([[0.0], body])


def distances(f: np.ndarray, S: int, K: int, g: np.ndarray) -> dict:
    """Eq. (13): d^2_ij for all 1-based i, j with |i - j| <= S, from Vbar."""
    n = len(f)
    Vb = filtered_V(f, S, K, g)
    out = {}
    for i in range(1, n + 1):
        for j in range(max(1, i - S), min(n, i + S) + 1):
            a, b = (i, j) if i >= j else (j, i)
            out[(i, j)] = Vb[packed_index(a, a, n, S, K)] + Vb[packed_index(b, b, n, S, K)] \
                - 2.0 * Vb[packed_index(a, b, n, S, K)]
    return out


def patchlift_nlm(f: np.ndarray, S: int, K: int, h: float, g: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Alg. 2 on the (already extended) signal f, for 0-based centres lo..hi-1
    whose patches and windows stay inside f."""
    d = distances(f, S, K, g)
    out = np.empty(hi - lo)
    for c in range(lo, hi):
        i = c + 1
        P = Q = 0.0
        for j in range(i - S, i + S + 1):
            w = np.exp(-d[(i, j)] / (h * h))
            P += w * f[j - 1]
            Q += w
        out[c - lo] = P / Q
    return out


def extend(f: np.ndarray, R: int) -> np.ndarray:
    """Half-sample symmetric extension by R samples per side (numpy's 'symmetric' pad)."""
    return np.pad(np.asarray(f, np.float64), R, mode="symmetric")
