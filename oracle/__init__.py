"""FP64 CPU oracle for separable non-local means (Ghosh & Chaudhury, arXiv:1407.2343).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package. The product
path (``paper_1407_2343_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``snlm_oracle.c`` (plain C, double precision, explicit
(2K+1)-tap patch sums, one pixel at a time); this module builds it with gcc and
wraps it with ctypes. Inputs are the exact stored sample values converted to
float64 by the caller; outputs are float64.

Functions and the passages they follow:
  ext_index      half-sample symmetric extension (boundary reading, Sec. II)
  profile        g_beta of Sec. II (box or Gaussian, Eq. (3))
  iir_coeffs     the recursive Gaussian of Young and van Vliet (1995) that Sec. II-B
                 names for the constant-time Gaussian profile: B, b1/b0, b2/b0, b3/b0, q
  iir_margin     samples outside a line at which its two passes start from rest
  iir_filter     that filter (causal then anti-causal pass) of a finite sequence
  default_h      h = sigma * sqrt(sum_k g(k))
  patch_dist_1d  Eq. (3) for every i and every offset s in [-S, S]
  nlm_1d         Eq. (4) and, when asked, the divergence of Eq. (24) (Alg. 3)
  snlm           Alg. 4 with Eqs. (14), (19), (25); orders RC, CR, AVG, SURE
  snlm_parts     the intermediate images and derivative maps of Alg. 4
  nlm_2d         the 2-D non-local means of Eqs. (1)-(2) (the comparison workload)
  snlm_3d        the separable 3-D extension: Eq. (4) along each axis of a volume in turn
  bf_params      sigma_s and sigma_r of the bilateral post-filter (Sec. IV-A)
  bilateral      the bilateral post-filter, Eq. (BF) of Sec. III-B
  snlm_full      SNLM[f]: Alg. 4 followed by the bilateral post-filter (Sec. III-B)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snlm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

BOX, GAUSS, GAUSS_IIR = 0, 1, 2
RC, CR, AVG, SURE = 0, 1, 2, 3
ORDERS = {"RC": RC, "CR": CR, "AVG": AVG, "SURE": SURE}
PROFILES = {"box": BOX, "gauss": GAUSS, "BOX": BOX, "GAUSS": GAUSS, "gauss_iir": GAUSS_IIR,
            "GAUSS_IIR": GAUSS_IIR}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        i64, ci, cd = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_ext.argtypes = [i64, i64]
        lib.orc_ext.restype = i64
        lib.orc_profile.argtypes = [ci, ci, cd, dp]
        lib.orc_profile.restype = None
        lib.orc_default_h.argtypes = [cd, ci, ci, cd]
        lib.orc_default_h.restype = cd
        lib.orc_iir_coeffs.argtypes = [cd, dp]
        lib.orc_iir_coeffs.restype = ci
        lib.orc_iir_margin.argtypes = [cd]
        lib.orc_iir_margin.restype = i64
        lib.orc_iir_filter.argtypes = [dp, i64, cd, dp]
        lib.orc_iir_filter.restype = ci
        lib.orc_patch_dist_1d.argtypes = [dp, i64, i64, ci, ci, ci, cd, dp, ci]
        lib.orc_patch_dist_1d.restype = ci
        lib.orc_nlm_1d.argtypes = [dp, i64, i64, ci, ci, cd, ci, cd, dp, dp, dp, ci]
        lib.orc_nlm_1d.restype = ci
        lib.orc_snlm.argtypes = [dp, i64, i64, ci, ci, cd, ci, cd, ci, cd, dp, dp, ci]
        lib.orc_snlm.restype = ci
        lib.orc_snlm_parts.argtypes = [dp, i64, i64, ci, ci, cd, ci, cd, dp, dp, dp, dp, dp, dp, ci]
        lib.orc_snlm_parts.restype = ci
        lib.orc_nlm_2d.argtypes = [dp, i64, i64, ci, ci, ci, ci, cd, ci, cd, dp, ci]
        lib.orc_nlm_2d.restype = ci
        lib.orc_bf_params.argtypes = [cd, dp, dp]
        lib.orc_bf_params.restype = None
        lib.orc_bilateral.argtypes = [dp, i64, i64, cd, cd, dp, ci]
        lib.orc_bilateral.restype = ci
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = ci
        _lib = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _nt(nthreads):
    return int(nthreads) if nthreads else _load().orc_max_threads()


def _profile_id(p):
    return PROFILES[p] if isinstance(p, str) else int(p)


def _order_id(o):
    return ORDERS[o] if isinstance(o, str) else int(o)


def default_beta(K: int) -> float:
    """Gaussian width used when none is given: beta = K/2 (K = 0 gives a delta)."""
    return max(K / 2.0, 1e-3)


def ext_index(x: int, N: int) -> int:
    return int(_load().orc_ext(int(x), int(N)))


def profile(K: int, prof="box", beta: float | None = None) -> np.ndarray:
    g = np.empty(2 * K + 1, np.float64)
    _load().orc_profile(K, _profile_id(prof), float(beta if beta is not None else default_beta(K)), _ptr(g))
    return g


def iir_coeffs(beta: float) -> dict:
    """Young-van Vliet coefficients for standard deviation beta (0.5 <= beta <= 64)."""
    c = np.empty(5, np.float64)
    if _load().orc_iir_coeffs(float(beta), _ptr(c)) != 0:
        raise ValueError(f"recursive Gaussian needs 0.5 <= beta <= 64 (got {beta})")
    return dict(zip(("B", "a1", "a2", "a3", "q"), c.tolist()))


def iir_margin(beta: float) -> int:
    m = int(_load().orc_iir_margin(float(beta)))
    if m < 0:
        raise ValueError(f"recursive Gaussian needs 0.5 <= beta <= 64 (got {beta})")
    return m


def iir_filter(x, beta: float) -> np.ndarray:
    """The recursive Gaussian (causal, then anti-causal pass) of a 1-D sequence,
    from a zero state outside it."""
    xv = _f64(x).ravel()
    y = np.empty_like(xv)
    if _load().orc_iir_filter(_ptr(xv), xv.size, float(beta), _ptr(y)) != 0:
        raise ValueError(f"recursive Gaussian needs 0.5 <= beta <= 64 (got {beta})")
    return y


def default_h(sigma: float, K: int, prof="box", beta: float | None = None) -> float:
    return float(_load().orc_default_h(float(sigma), int(K), _profile_id(prof),
                                       float(beta if beta is not None else default_beta(K))))


def patch_dist_1d(lines, S: int, K: int, prof="box", beta: float | None = None, nthreads: int = 0):
    """lines: (n, N) array -> (n, N, 2S+1) squared distances d^2(i, i+s) (Eq. (3))."""
    x = _f64(lines)
    if x.ndim == 1:
        x = x[None]
    n, N = x.shape
    out = np.empty((n, N, 2 * S + 1), np.float64)
    rc = _load().orc_patch_dist_1d(_ptr(x), n, N, S, K, _profile_id(prof),
                                   float(beta if beta is not None else default_beta(K)), _ptr(out), _nt(nthreads))
    if rc != 0:
        raise ValueError(f"oracle patch_dist_1d rejected its arguments (rc={rc})")
    return out


def nlm_1d(lines, S: int, K: int, h: float, prof="box", beta: float | None = None,
           delta_in=None, with_delta: bool = False, nthreads: int = 0):
    """Eq. (4) on each row of `lines` (n, N). Returns fhat, or (fhat, delta_out)."""
    x = _f64(lines)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[None]
    n, N = x.shape
    fh = np.empty_like(x)
    din = None if delta_in is None else _f64(delta_in).reshape(n, N)
    dout = np.empty_like(x) if (with_delta or delta_in is not None) else None
    rc = _load().orc_nlm_1d(_ptr(x), n, N, S, K, float(h), _profile_id(prof),
                            float(beta if beta is not None else default_beta(K)),
                            _ptr(din), _ptr(fh), _ptr(dout), _nt(nthreads))
    if rc != 0:
        raise ValueError(f"oracle nlm_1d rejected its arguments (rc={rc})")
    if squeeze:
        fh = fh[0]
        dout = None if dout is None else dout[0]
    return (fh, dout) if dout is not None else fh


def snlm(img, S: int, K: int, h: float, prof="box", beta: float | None = None, order="RC",
         sigma: float = 0.0, nthreads: int = 0):
    """Alg. 4 on an (H, W) image. Returns (out, info) with info a dict of the
    combination weights and the sums of Eqs. (19) and (25)."""
    x = _f64(img)
    H, W = x.shape
    out = np.empty_like(x)
    info = np.zeros(10, np.float64)
    rc = _load().orc_snlm(_ptr(x), H, W, S, K, float(h), _profile_id(prof),
                          float(beta if beta is not None else default_beta(K)), _order_id(order),
                          float(sigma), _ptr(out), _ptr(info), _nt(nthreads))
    if rc != 0:
        raise ValueError(f"oracle snlm rejected its arguments (rc={rc})")
    keys = ["theta1", "theta2", "A11", "A12", "A22", "sum_f_frc", "sum_f_fcr", "sum_d1", "sum_d2", "sigma2"]
    return out, dict(zip(keys, info.tolist()))


def snlm_parts(img, S: int, K: int, h: float, prof="box", beta: float | None = None, nthreads: int = 0):
    """The intermediate results of Alg. 4: dict with fr, frc, fc, fcr, d1, d2."""
    x = _f64(img)
    H, W = x.shape
    parts = {k: np.empty_like(x) for k in ("fr", "frc", "fc", "fcr", "d1", "d2")}
    rc = _load().orc_snlm_parts(_ptr(x), H, W, S, K, float(h), _profile_id(prof),
                                float(beta if beta is not None else default_beta(K)),
                                *[_ptr(parts[k]) for k in ("fr", "frc", "fc", "fcr", "d1", "d2")],
                                _nt(nthreads))
    if rc != 0:
        raise ValueError(f"oracle snlm_parts rejected its arguments (rc={rc})")
    return parts


def nlm_2d(img, S, K, h: float, prof="box", alpha: float | None = None, nthreads: int = 0):
    """Eqs. (1)-(2) on an (H, W) image. S and K are ints (square window and patch) or
    (Sy, Sx) / (Ky, Kx) pairs; alpha defaults to K/2 (the larger K)."""
    x = _f64(img)
    H, W = x.shape
    Sy, Sx = (S, S) if np.isscalar(S) else S
    Ky, Kx = (K, K) if np.isscalar(K) else K
    out = np.empty_like(x)
    a = float(alpha if alpha is not None else default_beta(max(Ky, Kx)))
    rc = _load().orc_nlm_2d(_ptr(x), H, W, int(Sy), int(Sx), int(Ky), int(Kx), float(h), _profile_id(prof), a,
                            _ptr(out), _nt(nthreads))
    if rc != 0:
        raise ValueError(f"oracle nlm_2d rejected its arguments (rc={rc})")
    return out


def snlm_3d(vol, S: int, K: int, h: float, prof="box", beta: float | None = None, order="XYZ", nthreads: int = 0):
    """The separable 3-D extension of a (D, H, W) volume: the 1-D NLM of Eq. (4)
    along x (the last axis), y and z in the given order ("XYZ", any permutation of
    the three letters, or "AVG6", the average of the six orders), each pass on the
    previous pass's output."""
    x = _f64(vol)
    if order == "AVG6":
        orders = ["XYZ", "XZY", "YXZ", "YZX", "ZXY", "ZYX"]
        return sum(snlm_3d(x, S, K, h, prof, beta, o, nthreads) for o in orders) / 6.0
    axis_of = {"X": 2, "Y": 1, "Z": 0}
    for letter in order:
        ax = axis_of[letter]
        moved = np.moveaxis(x, ax, -1)
        shp = moved.shape
        f = nlm_1d(moved.reshape(-1, shp[-1]), S, K, h, prof, beta, nthreads=nthreads)
        x = np.moveaxis(np.asarray(f).reshape(shp), -1, ax)
    return np.ascontiguousarray(x)


def default_h_2d(sigma: float, K: int, prof="box", alpha: float | None = None) -> float:
    """h = sigma * sqrt(sum_k G(k)) over the (2K+1)^2 patch (the 2-D form of the 1-D rule)."""
    g = profile(K, prof, alpha)
    return float(sigma * np.sqrt(g.sum() ** 2))


def bf_params(sigma: float):
    """(sigma_s, sigma_r) of the bilateral post-filter for noise level sigma (Sec. IV-A)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _load().orc_bf_params(float(sigma), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def bilateral(img, sigma_s: float, sigma_r: float, nthreads: int = 0):
    """Eq. (BF) of Sec. III-B on an (H, W) image (support [-3 sigma_s, 3 sigma_s]^2)."""
    x = _f64(img)
    H, W = x.shape
    out = np.empty_like(x)
    rc = _load().orc_bilateral(_ptr(x), H, W, float(sigma_s), float(sigma_r), _ptr(out), _nt(nthreads))
    if rc != 0:
        raise ValueError(f"oracle bilateral rejected its arguments (rc={rc})")
    return out


def snlm_full(img, S: int, K: int, h: float, prof="box", beta: float | None = None, order="SURE",
              sigma: float = 0.0, sigma_s: float | None = None, sigma_r: float | None = None, nthreads: int = 0):
    """SNLM[f] of Sec. III-B: Alg. 4, then the bilateral post-filter (its parameters
    from the rules of Sec. IV-A unless given)."""
    ss, sr = bf_params(sigma)
    ft, _ = snlm(img, S, K, h, prof, beta, order=order, sigma=sigma, nthreads=nthreads)
    return bilateral(ft, ss if sigma_s is None else sigma_s, sr if sigma_r is None else sigma_r, nthreads)


def max_threads() -> int:
    return int(_load().orc_max_threads())
