"""Python binding of libsnlm with the C ABI's names (argument marshalling only).

Every function forwards to the entry point of the same name in libsnlm.so; all
computation runs in the library's CUDA kernels. Device buffers are PyTorch CUDA
tensors (used only for memory and streams); the current torch stream is used
unless one is given.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

U8, F16, F32 = 0, 1, 2
BOX, GAUSS, GAUSS_IIR = 0, 1, 2
RC, CR, AVG, SURE = 0, 1, 2, 3
OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_CHECK = 0, -1, -2, -3, -4, -5, -6
MAX_K, MAX_S = 7, 128

_ORDERS = {"RC": RC, "CR": CR, "AVG": AVG, "SURE": SURE}
_PROFILES = {"box": BOX, "gauss": GAUSS, "gauss_iir": GAUSS_IIR}


class SnlmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {snlm_status_str(status)} ({status})")


def _check(rc: int, where: str):
    if rc != OK:
        raise SnlmError(rc, where)


def _order(o):
    return _ORDERS[o.upper()] if isinstance(o, str) else int(o)


def _profile(p):
    return _PROFILES[p.lower()] if isinstance(p, str) else int(p)


def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    m = {torch.uint8: U8, torch.float16: F16, torch.float32: F32}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}; use uint8, float16 or float32")
    return m[t.dtype]


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def snlm_status_str(status: int) -> str:
    return _lib.load().snlm_status_str(int(status)).decode()


def snlm_version() -> int:
    return int(_lib.load().snlm_version())


KERNEL_COUNT = 234   # SNLM_KERNEL_COUNT of include/snlm.h


def snlm_preload() -> int:
    """Load every kernel of the library on the current device (see include/snlm.h);
    returns how many were loaded."""
    n = ctypes.c_int(0)
    _check(_lib.load().snlm_preload(ctypes.byref(n)), "snlm_preload")
    return int(n.value)


def snlm_default_h(sigma: float, K: int, profile="box", beta: float = 0.0) -> float:
    return float(_lib.load().snlm_default_h(float(sigma), int(K), _profile(profile), float(beta or 0.0)))


def snlm_workspace_bytes(H: int, W: int, order="RC") -> int:
    return int(_lib.load().snlm_workspace_bytes(int(H), int(W), _order(order)))


def _image_args(img):
    if img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("img must be a 2-D tensor with unit column stride")
    H, W = img.shape
    return _dtype_code(img), int(H), int(W), int(img.stride(0))


def _h_for(h, sigma, K, profile, beta):
    if h is None:
        if sigma is None:
            raise ValueError("give h or sigma")
        h = snlm_default_h(sigma, K, profile, beta or 0.0)
    return float(h)


def snlm_denoise(img, S: int, K: int, h: float | None = None, profile="box", order="RC",
                 sigma: float | None = None, beta: float = 0.0, out=None, stream=None):
    """Separable NLM of one device image (Alg. 4 without the bilateral
    post-filter). Returns the float32 (H, W) output tensor."""
    torch = _torch()
    dt, H, W, pitch = _image_args(img)
    h = _h_for(h, sigma, K, profile, beta)
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    rc = _lib.load().snlm_denoise(_ptr(img), dt, H, W, pitch, int(S), int(K), h, _profile(profile),
                                  _order(order), float(sigma or 0.0), float(beta or 0.0), _ptr(out),
                                  _stream_ptr(stream))
    _check(rc, "snlm_denoise")
    return out


def snlm_denoise_ws(img, S: int, K: int, h: float | None = None, profile="box", order="RC",
                    sigma: float | None = None, beta: float = 0.0, out=None, workspace=None,
                    info=None, stream=None):
    """As snlm_denoise with caller-provided scratch (a uint8 CUDA tensor of at
    least snlm_workspace_bytes bytes) and an optional float64 `info` tensor (10)."""
    torch = _torch()
    dt, H, W, pitch = _image_args(img)
    h = _h_for(h, sigma, K, profile, beta)
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    if workspace is None:
        workspace = torch.empty(snlm_workspace_bytes(H, W, order), dtype=torch.uint8, device=img.device)
    rc = _lib.load().snlm_denoise_ws(_ptr(img), dt, H, W, pitch, int(S), int(K), h, _profile(profile),
                                     _order(order), float(sigma or 0.0), float(beta or 0.0), _ptr(out),
                                     _ptr(workspace), int(workspace.numel() * workspace.element_size()),
                                     _ptr(info), _stream_ptr(stream))
    _check(rc, "snlm_denoise_ws")
    return out


def snlm_denoise_host(img: np.ndarray, S: int, K: int, h: float | None = None, profile="box",
                      order="RC", sigma: float | None = None, beta: float = 0.0, out: np.ndarray | None = None,
                      stream=None) -> np.ndarray:
    """End-to-end call on HOST arrays (numpy or pinned CPU tensors): copy in,
    denoise, copy out; returns when the result is in `out`."""
    torch = _torch()
    if isinstance(img, np.ndarray):
        codes = {np.dtype(np.uint8): U8, np.dtype(np.float16): F16, np.dtype(np.float32): F32}
        if img.ndim != 2 or img.dtype not in codes:
            raise TypeError("img must be a 2-D uint8/float16/float32 array")
        a = np.ascontiguousarray(img)
        dt, (H, W), pitch, iptr = codes[a.dtype], a.shape, a.shape[1], ctypes.c_void_p(a.ctypes.data)
        keep = a
    else:
        dt, H, W, pitch = _image_args(img)
        iptr, keep = _ptr(img), img
    h = _h_for(h, sigma, K, profile, beta)
    if out is None:
        out = np.empty((H, W), np.float32)
    optr = ctypes.c_void_p(out.ctypes.data) if isinstance(out, np.ndarray) else _ptr(out)
    rc = _lib.load().snlm_denoise_host(iptr, dt, H, W, pitch, int(S), int(K), h, _profile(profile),
                                       _order(order), float(sigma or 0.0), float(beta or 0.0), optr,
                                       _stream_ptr(stream) if torch.cuda.is_available() else None)
    del keep
    _check(rc, "snlm_denoise_host")
    return out


def snlm_denoise_host_many(imgs, S: int, K: int, h: float | None = None, profile="box", order="RC",
                           sigma: float | None = None, beta: float = 0.0, outs=None, stream=None):
    """Pipelined end-to-end call on a sequence of same-shaped HOST images (numpy
    arrays or CPU tensors, pinned for the overlap): each is copied in, denoised and
    copied out as by snlm_denoise_host, with the copies overlapped with the
    neighbours' computation. Returns the list of outputs (float32, H x W)."""
    torch = _torch()
    imgs = list(imgs)
    if not imgs:
        return []
    codes = {np.dtype(np.uint8): U8, np.dtype(np.float16): F16, np.dtype(np.float32): F32}
    keep, ptrs, shape = [], [], None
    for im in imgs:
        if isinstance(im, np.ndarray):
            if im.ndim != 2 or im.dtype not in codes:
                raise TypeError("images must be 2-D uint8/float16/float32 arrays")
            a = np.ascontiguousarray(im)
            args = (codes[a.dtype], a.shape[0], a.shape[1], a.shape[1])
            ptrs.append(a.ctypes.data)
            keep.append(a)
        else:
            args = _image_args(im)
            ptrs.append(_ptr(im).value)
            keep.append(im)
        if shape is None:
            shape = args
        elif args != shape:
            raise ValueError("all images must have the same dtype, shape and pitch")
    dt, H, W, pitch = shape
    h = _h_for(h, sigma, K, profile, beta)
    if outs is None:
        outs = [np.empty((H, W), np.float32) for _ in imgs]
    if len(outs) != len(imgs):
        raise ValueError("one output per image")
    for o in outs:
        ok = o.shape == (H, W) and (o.dtype == np.float32 and o.flags.c_contiguous if isinstance(o, np.ndarray)
                                    else o.dtype == torch.float32 and o.is_contiguous() and o.device.type == "cpu")
        if not ok:
            raise ValueError("outputs must be contiguous float32 host arrays of shape (H, W)")
    optrs = [o.ctypes.data if isinstance(o, np.ndarray) else _ptr(o).value for o in outs]
    n = len(imgs)
    iarr = (ctypes.c_void_p * n)(*ptrs)
    oarr = (ctypes.c_void_p * n)(*optrs)
    rc = _lib.load().snlm_denoise_host_many(iarr, oarr, n, dt, H, W, pitch, int(S), int(K), h, _profile(profile),
                                            _order(order), float(sigma or 0.0), float(beta or 0.0),
                                            _stream_ptr(stream) if torch.cuda.is_available() else None)
    del keep
    _check(rc, "snlm_denoise_host_many")
    return outs


def snlm_bf_params(sigma: float):
    """(sigma_s, sigma_r) of the bilateral post-filter for noise level sigma (Sec. IV-A)."""
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(_lib.load().snlm_bf_params(float(sigma), ctypes.byref(a), ctypes.byref(b)), "snlm_bf_params")
    return a.value, b.value


def snlm_bilateral(x, sigma_s: float, sigma_r: float, out=None, stream=None):
    """Bilateral post-filter of Sec. III-B (Eq. (BF)) of a 2-D float32 device tensor
    with unit column stride; returns out (float32, contiguous unless given)."""
    torch = _torch()
    if x.dim() != 2 or x.dtype != torch.float32 or x.stride(1) != 1:
        raise ValueError("x must be a 2-D float32 tensor with unit column stride")
    H, W = x.shape
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=x.device)
    if out.shape != x.shape or out.dtype != torch.float32 or out.stride(1) != 1:
        raise ValueError("out must be float32 with x's shape and unit column stride")
    rc = _lib.load().snlm_bilateral(_ptr(x), int(H), int(W), int(x.stride(0)), float(sigma_s), float(sigma_r),
                                    _ptr(out), int(out.stride(0)), _stream_ptr(stream))
    _check(rc, "snlm_bilateral")
    return out


def snlm_denoise_bf(img, S: int, K: int, h: float | None = None, profile="box", order="SURE",
                    sigma: float | None = None, beta: float = 0.0, sigma_s: float = 0.0, sigma_r: float = 0.0,
                    out=None, stream=None):
    """SNLM[f] of Sec. III-B: Alg. 4, then the bilateral post-filter (its parameters
    from the rules of Sec. IV-A when sigma_s or sigma_r is <= 0)."""
    torch = _torch()
    dt, H, W, pitch = _image_args(img)
    h = _h_for(h, sigma, K, profile, beta)
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    if out.shape != (H, W) or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 (H, W) tensor")
    rc = _lib.load().snlm_denoise_bf(_ptr(img), dt, H, W, pitch, int(S), int(K), h, _profile(profile),
                                     _order(order), float(sigma or 0.0), float(beta or 0.0), float(sigma_s),
                                     float(sigma_r), _ptr(out), _stream_ptr(stream))
    _check(rc, "snlm_denoise_bf")
    return out


def snlm_nlm_2d(img, S: int, K: int, h: float, profile="box", alpha: float = 0.0, out=None, stream=None):
    """The 2-D non-local means of Eqs. (1)-(2) of a 2-D device tensor (uint8,
    float16 or float32, unit column stride); returns out (float32, contiguous)."""
    torch = _torch()
    dt, H, W, pitch = _image_args(img)
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    if out.shape != (H, W) or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 (H, W) tensor")
    rc = _lib.load().snlm_nlm_2d(_ptr(img), dt, H, W, pitch, int(S), int(K), float(h), _profile(profile),
                                 float(alpha or 0.0), _ptr(out), _stream_ptr(stream))
    _check(rc, "snlm_nlm_2d")
    return out


ORDERS3 = {"XYZ": 0, "AVG6": 1}


def snlm_denoise_3d(vol, S: int, K: int, h: float, profile="box", beta: float = 0.0, order3="XYZ", out=None,
                    stream=None):
    """Separable 3-D extension: the 1-D pass along x, y and z of a dense (D, H, W)
    device tensor (uint8, float16 or float32); order3 "XYZ" or "AVG6" (the average
    of the six orders). Returns out (float32, (D, H, W))."""
    torch = _torch()
    if vol.dim() != 3 or not vol.is_contiguous():
        raise ValueError("vol must be a contiguous 3-D tensor (D, H, W)")
    D, H, W = vol.shape
    if out is None:
        out = torch.empty((D, H, W), dtype=torch.float32, device=vol.device)
    if out.shape != vol.shape or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 tensor of vol's shape")
    rc = _lib.load().snlm_denoise_3d(_ptr(vol), _dtype_code(vol), int(D), int(H), int(W), int(S), int(K), float(h),
                                     _profile(profile), float(beta or 0.0), ORDERS3[order3] if isinstance(order3, str)
                                     else int(order3), _ptr(out), _stream_ptr(stream))
    _check(rc, "snlm_denoise_3d")
    return out


def snlm_nlm_1d(x, S: int, K: int, h: float, profile="box", beta: float = 0.0, fhat=None,
                delta_in=None, delta_out=None, stream=None):
    """One 1-D NLM pass (Eq. (4)) over the rows of a 2-D device tensor `x`
    (n_lines, N) with arbitrary strides; returns fhat (float32, contiguous)."""
    torch = _torch()
    if x.dim() != 2:
        raise ValueError("x must be 2-D (n_lines, N)")
    n, N = x.shape
    if fhat is None:
        fhat = torch.empty((n, N), dtype=torch.float32, device=x.device)
    for t in (delta_in, delta_out):
        if t is not None and (t.shape != fhat.shape or t.stride() != fhat.stride() or t.dtype != torch.float32):
            raise ValueError("delta tensors must be float32 with fhat's shape and strides")
    rc = _lib.load().snlm_nlm_1d(_ptr(x), _dtype_code(x), int(n), int(N), int(x.stride(0)), int(x.stride(1)),
                                 int(S), int(K), float(h), _profile(profile), float(beta or 0.0), _ptr(fhat),
                                 int(fhat.stride(0)), int(fhat.stride(1)), _ptr(delta_in), _ptr(delta_out),
                                 _stream_ptr(stream))
    _check(rc, "snlm_nlm_1d")
    return fhat


def snlm_patch_dist_1d(x, S: int, K: int, profile="box", beta: float = 0.0, out=None, stream=None):
    """Patch distances (Eq. (3)) of the rows of a 2-D device tensor (n, N):
    returns (n, N, 2S+1), int32 for uint8 input with the box profile else float32."""
    torch = _torch()
    if x.dim() != 2 or x.stride(1) != 1:
        raise ValueError("x must be 2-D with unit stride along lines")
    n, N = x.shape
    as_int = x.dtype == torch.uint8 and _profile(profile) == BOX
    if out is None:
        out = torch.empty((n, N, 2 * S + 1), dtype=torch.int32 if as_int else torch.float32, device=x.device)
    rc = _lib.load().snlm_patch_dist_1d(_ptr(x), _dtype_code(x), int(n), int(N), int(x.stride(0)), int(S),
                                        int(K), _profile(profile), float(beta or 0.0), _ptr(out),
                                        _stream_ptr(stream))
    _check(rc, "snlm_patch_dist_1d")
    return out


def snlm_trace_enable(enable: bool = True) -> bool:
    """Bracket every library kernel launch with CUDA events (process-wide)."""
    return bool(_lib.load().snlm_trace_enable(1 if enable else 0))


def snlm_trace_read(max_records: int = 1 << 16):
    """Per-launch device times since the last read: list of (kernel_name, ms)."""
    lib = _lib.load()
    kinds = (ctypes.c_int * max_records)()
    ms = (ctypes.c_float * max_records)()
    n = ctypes.c_int(0)
    _check(lib.snlm_trace_read(kinds, ms, max_records, ctypes.byref(n)), "snlm_trace_read")
    return [(lib.snlm_kernel_name(kinds[i]).decode(), float(ms[i])) for i in range(n.value)]


def snlm_kernel_name(kind: int) -> str:
    return _lib.load().snlm_kernel_name(int(kind)).decode()


def snlm_probe_peaks(stream=None) -> dict:
    """Measured FP32 (packed FP32x2 and scalar FMA) lane-operations/s and MUFU.EX2
    results/s of the current device (see include/snlm.h)."""
    rates = (ctypes.c_double * 3)()
    _check(_lib.load().snlm_probe_peaks(rates, _stream_ptr(stream)), "snlm_probe_peaks")
    return {"fp32_fma2_ops_s": rates[0], "fp32_fma_ops_s": rates[1], "ex2_s": rates[2]}


OPT_TMA, OPT_WAIT_LIMIT_US, OPT_INJECT_WAIT_TIMEOUT = 0, 1, 2


def snlm_set_option(option: int, value: int):
    _check(_lib.load().snlm_set_option(int(option), int(value)), "snlm_set_option")


def snlm_get_option(option: int) -> int:
    return int(_lib.load().snlm_get_option(int(option)))


def snlm_device_error(stream=None) -> int:
    """Wait for `stream`, return (and clear) the device-side failure record:
    OK, or ERR_TIMEOUT when a bounded wait of a TMA pass gave up."""
    return int(_lib.load().snlm_device_error(_stream_ptr(stream)))


def snlm_sure_band(img, S: int, K: int, h: float | None = None, profile="box", beta: float = 0.0, row0: int = 0,
                   row1: int | None = None, sigma: float | None = None, f_rc=None, f_cr=None, sums=None,
                   workspace=None, stream=None):
    """Alg. 4's four passes of `img` (a band with its halo rows, or a whole image)
    keeping f_rc and f_cr apart, and the seven SURE sums over rows [row0, row1) in
    the basis m = (f_rc + f_cr)/2, d = (f_rc - f_cr)/2 (see include/snlm.h).
    Returns (f_rc, f_cr, sums) with sums a float64 CUDA tensor of 7."""
    torch = _torch()
    dt, H, W, pitch = _image_args(img)
    h = _h_for(h, sigma, K, profile, beta)
    row1 = H if row1 is None else int(row1)
    f_rc = torch.empty((H, W), dtype=torch.float32, device=img.device) if f_rc is None else f_rc
    f_cr = torch.empty((H, W), dtype=torch.float32, device=img.device) if f_cr is None else f_cr
    sums = torch.empty(7, dtype=torch.float64, device=img.device) if sums is None else sums
    if workspace is None:
        workspace = torch.empty(snlm_workspace_bytes(H, W, "SURE"), dtype=torch.uint8, device=img.device)
    rc = _lib.load().snlm_sure_band(_ptr(img), dt, H, W, pitch, int(S), int(K), h, _profile(profile),
                                    float(beta or 0.0), int(row0), row1, _ptr(f_rc), _ptr(f_cr), _ptr(sums),
                                    _ptr(workspace), ctypes.c_size_t(workspace.numel()), _stream_ptr(stream))
    _check(rc, "snlm_sure_band")
    return f_rc, f_cr, sums


def snlm_sure_theta(sums, sigma: float):
    """theta = (theta1, theta2) of Eqs. (19), (25) from seven sums (host sequence)."""
    import numpy as np

    arr = (ctypes.c_double * 7)(*[float(x) for x in np.asarray(sums, dtype=np.float64).ravel()[:7]])
    th = (ctypes.c_double * 2)()
    _check(_lib.load().snlm_sure_theta(arr, float(sigma), th), "snlm_sure_theta")
    return float(th[0]), float(th[1])


def snlm_sure_combine(f_rc, f_cr, theta, out=None, stream=None):
    """out = theta1 f_rc + theta2 f_cr (device float32 tensors of the same shape)."""
    torch = _torch()
    if f_rc.shape != f_cr.shape or not f_rc.is_contiguous() or not f_cr.is_contiguous():
        raise ValueError("f_rc and f_cr must be contiguous tensors of one shape")
    out = torch.empty_like(f_rc) if out is None else out
    rc = _lib.load().snlm_sure_combine(_ptr(f_rc), _ptr(f_cr), int(f_rc.numel()), float(theta[0]),
                                       float(theta[1]), _ptr(out), _stream_ptr(stream))
    _check(rc, "snlm_sure_combine")
    return out


NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def snlm_denoise_noalloc(img, S: int, K: int, h: float | None = None, profile="box", order="RC",
                         sigma: float | None = None, beta: float = 0.0, out=None, stream=None):
    """snlm_denoise without any device allocation inside the library: the
    intermediate images use a fixed 32 MiB scratch area compiled into it. For
    callers that may not allocate device memory at run time; `out` should then be
    given (a new output tensor is allocated here only if it is not). Calls that can
    overlap on the GPU share the scratch area and must be serialised."""
    torch = _torch()
    dt, H, W, pitch = _image_args(img)
    h = _h_for(h, sigma, K, profile, beta)
    if out is None:
        out = torch.empty((H, W), dtype=torch.float32, device=img.device)
    rc = _lib.load().snlm_denoise_noalloc(_ptr(img), dt, H, W, pitch, int(S), int(K), h, _profile(profile),
                                          _order(order), float(sigma or 0.0), float(beta or 0.0), _ptr(out),
                                          _stream_ptr(stream))
    _check(rc, "snlm_denoise_noalloc")
    return out


# ---------------------------------------------------------------- batches


def _request(img, out, S, K, h, profile, order, sigma, beta):
    dt, H, W, pitch = _image_args(img)
    return _lib.Request(img.data_ptr(), out.data_ptr(), dt, H, W, pitch, int(S), int(K), float(h),
                        _profile(profile), _order(order), float(sigma or 0.0), float(beta or 0.0))


def snlm_batch_plan_create(requests, ctas_per_sm: int = 0, queue_order: int = 0, spin_limit_us: int = 0,
                           fail_job: int = -1):
    """Build a batch plan. `requests` is a list of dicts with keys img, out (CUDA
    tensors), S, K, h, and optionally profile, order, sigma, beta. Returns an opaque
    handle (int); keep the tensors alive while the plan is used."""
    arr = (_lib.Request * len(requests))()
    for i, r in enumerate(requests):
        arr[i] = _request(r["img"], r["out"], r["S"], r["K"], r["h"], r.get("profile", "box"),
                          r.get("order", "RC"), r.get("sigma", 0.0), r.get("beta", 0.0))
    cfg = _lib.BatchConfig(int(ctas_per_sm), int(queue_order), int(spin_limit_us), int(fail_job))
    h = ctypes.c_void_p()
    _check(_lib.load().snlm_batch_plan_create(arr, len(requests), ctypes.byref(cfg), ctypes.byref(h)),
           "snlm_batch_plan_create")
    return h.value


def snlm_batch_plan_workspace_bytes(plan) -> int:
    return int(_lib.load().snlm_batch_plan_workspace_bytes(ctypes.c_void_p(plan)))


def snlm_batch_plan_upload(plan, workspace, stream=None):
    _check(_lib.load().snlm_batch_plan_upload(ctypes.c_void_p(plan), _ptr(workspace),
                                              int(workspace.numel() * workspace.element_size()),
                                              _stream_ptr(stream)), "snlm_batch_plan_upload")


def snlm_batch_plan_launch(plan, stream=None):
    _check(_lib.load().snlm_batch_plan_launch(ctypes.c_void_p(plan), _stream_ptr(stream)),
           "snlm_batch_plan_launch")


def snlm_batch_plan_capture(plan, stream=None):
    _check(_lib.load().snlm_batch_plan_capture(ctypes.c_void_p(plan), _stream_ptr(stream)),
           "snlm_batch_plan_capture")


def snlm_batch_plan_status(plan, stream=None) -> int:
    """0 when the last run finished normally, ERR_TIMEOUT when a bounded wait gave up."""
    return int(_lib.load().snlm_batch_plan_status(ctypes.c_void_p(plan), _stream_ptr(stream)))


def snlm_batch_plan_status_async(plan, host_word, stream=None):
    """Enqueue a copy of the plan's failure word into `host_word` (a pinned int32
    host tensor of at least one element) on the stream, without waiting; nonzero
    there, once the stream has passed this point, means a bounded wait gave up."""
    if host_word.dtype != _torch().int32 or host_word.device.type != "cpu" or host_word.numel() < 1:
        raise ValueError("host_word must be an int32 host tensor with at least one element")
    _check(_lib.load().snlm_batch_plan_status_async(ctypes.c_void_p(plan), ctypes.c_void_p(host_word.data_ptr()),
                                                    _stream_ptr(stream)), "snlm_batch_plan_status_async")


def snlm_batch_plan_info(plan):
    j, u, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib.load().snlm_batch_plan_info(ctypes.c_void_p(plan), ctypes.byref(j), ctypes.byref(u),
                                            ctypes.byref(c)), "snlm_batch_plan_info")
    return {"jobs": j.value, "units": u.value, "classes": c.value}


def snlm_batch_plan_destroy(plan):
    _lib.load().snlm_batch_plan_destroy(ctypes.c_void_p(plan))


# ------------------------------------------------------------------ serving loop

SERVE_BATCHED, SERVE_PLAIN = 0, 1


def snlm_server_create(mode: int = SERVE_BATCHED, mem_budget: int = 0, streams: int = 4, max_batch: int = 256,
                       solo_pixels: int = 1 << 20, ctas_per_sm: int = 0):
    """Create a serving loop (see include/snlm.h); returns its handle."""
    lib = _lib.load()
    cfg = _lib.ServerConfig(int(mode), int(mem_budget), int(streams), int(max_batch), int(solo_pixels),
                            int(ctas_per_sm))
    h = ctypes.c_void_p()
    _check(lib.snlm_server_create(ctypes.byref(cfg), ctypes.byref(h)), "snlm_server_create")
    return h.value


def snlm_server_submit(server, requests):
    """Queue requests: dicts with img and out (pinned CPU tensors), S, K, h,
    profile, order, sigma, beta, t_arrival. Returns their ids."""
    lib = _lib.load()
    n = len(requests)
    arr = (_lib.ServeRequest * n)()
    for i, r in enumerate(requests):
        dt, H, W, pitch = _image_args(r["img"])
        arr[i] = _lib.ServeRequest(r["img"].data_ptr(), r["out"].data_ptr(), dt, H, W, pitch, int(r["S"]),
                                   int(r["K"]), float(r["h"]), _profile(r.get("profile", "box")),
                                   _order(r.get("order", "RC")), float(r.get("sigma") or 0.0),
                                   float(r.get("beta") or 0.0), float(r["t_arrival"]))
    ids = (ctypes.c_int * max(n, 1))()
    _check(lib.snlm_server_submit(ctypes.c_void_p(server), arr, n, ids), "snlm_server_submit")
    return [ids[i] for i in range(n)]


def snlm_server_drain(server):
    _check(_lib.load().snlm_server_drain(ctypes.c_void_p(server)), "snlm_server_drain")


def snlm_server_result(server, rid: int):
    """(completion time on the server clock, launch index) of a request."""
    t, k = ctypes.c_double(), ctypes.c_int()
    _check(_lib.load().snlm_server_result(ctypes.c_void_p(server), int(rid), ctypes.byref(t), ctypes.byref(k)),
           "snlm_server_result")
    return t.value, k.value


def snlm_server_get_stats(server) -> dict:
    st = _lib.ServerStats()
    _check(_lib.load().snlm_server_get_stats(ctypes.c_void_p(server), ctypes.byref(st)), "snlm_server_get_stats")
    return {name: getattr(st, name) for name, _ in st._fields_}


def snlm_server_clock(server) -> float:
    return float(_lib.load().snlm_server_clock(ctypes.c_void_p(server)))


def snlm_server_destroy(server):
    if server:
        _lib.load().snlm_server_destroy(ctypes.c_void_p(server))

