"""ctypes declarations of libsnlm's C ABI (include/snlm.h).

The shared library is built in-tree by ``paper_1407_2343_gb300.build`` and loaded
from this package directory. There is no fallback: if the library is missing,
every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
# SNLM_LIBRARY selects another build of the library (the checked build in tests)
LIB_PATH = os.environ.get("SNLM_LIBRARY") or os.path.join(_PKG, "libsnlm.so")

_lock = threading.Lock()
_lib = None


class LibraryMissing(RuntimeError):
    pass


class Request(ctypes.Structure):
    """snlm_request of include/snlm.h."""
    _fields_ = [("img", ctypes.c_void_p), ("out", ctypes.c_void_p), ("dtype", ctypes.c_int),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("pitch", ctypes.c_int), ("S", ctypes.c_int),
                ("K", ctypes.c_int), ("h", ctypes.c_float), ("profile", ctypes.c_int), ("order", ctypes.c_int),
                ("sigma", ctypes.c_float), ("beta", ctypes.c_float)]


class BatchConfig(ctypes.Structure):
    """snlm_batch_config of include/snlm.h."""
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("queue_order", ctypes.c_int),
                ("spin_limit_us", ctypes.c_int), ("fail_job", ctypes.c_int)]


class ServeRequest(ctypes.Structure):
    """snlm_serve_request of include/snlm.h."""
    _fields_ = [("img", ctypes.c_void_p), ("out", ctypes.c_void_p), ("dtype", ctypes.c_int),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("pitch", ctypes.c_int), ("S", ctypes.c_int),
                ("K", ctypes.c_int), ("h", ctypes.c_float), ("profile", ctypes.c_int), ("order", ctypes.c_int),
                ("sigma", ctypes.c_float), ("beta", ctypes.c_float), ("t_arrival", ctypes.c_double)]


class ServerConfig(ctypes.Structure):
    """snlm_server_config of include/snlm.h."""
    _fields_ = [("mode", ctypes.c_int), ("mem_budget", ctypes.c_longlong), ("streams", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("solo_pixels", ctypes.c_longlong), ("ctas_per_sm", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    """snlm_server_stats of include/snlm.h."""
    _fields_ = [("launches", ctypes.c_int), ("max_batch", ctypes.c_int), ("max_inflight", ctypes.c_int),
                ("images", ctypes.c_int), ("max_used_bytes", ctypes.c_longlong),
                ("budget_bytes", ctypes.c_longlong), ("wall_s", ctypes.c_double), ("host_busy_s", ctypes.c_double),
                ("max_yield_s", ctypes.c_double), ("max_iter_s", ctypes.c_double), ("yields_over_1ms", ctypes.c_int)]


def load(build_if_missing: bool = False):
    """Load libsnlm.so (optionally building it first). Raises LibraryMissing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise LibraryMissing(
                    f"{LIB_PATH} is not built; run `python -m paper_1407_2343_gb300.build` "
                    "(needs nvcc). There is no CPU fallback.")
            from . import build as _b
            _b.build()
        lib = ctypes.CDLL(LIB_PATH)
        vp, ci, cf, cll, csz, dp = (ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong,
                                    ctypes.c_size_t, ctypes.POINTER(ctypes.c_double))
        fp = ctypes.POINTER(ctypes.c_float)
        lib.snlm_status_str.argtypes = [ci]
        lib.snlm_status_str.restype = ctypes.c_char_p
        lib.snlm_version.argtypes = []
        lib.snlm_version.restype = ci
        lib.snlm_preload.argtypes = [ctypes.POINTER(ci)]
        lib.snlm_preload.restype = ci
        lib.snlm_default_h.argtypes = [cf, ci, ci, cf]
        lib.snlm_default_h.restype = cf
        lib.snlm_workspace_bytes.argtypes = [ci, ci, ci]
        lib.snlm_workspace_bytes.restype = csz
        lib.snlm_denoise.argtypes = [vp, ci, ci, ci, ci, ci, ci, cf, ci, ci, cf, cf, vp, vp]
        lib.snlm_denoise.restype = ci
        lib.snlm_denoise_ws.argtypes = [vp, ci, ci, ci, ci, ci, ci, cf, ci, ci, cf, cf, vp, vp, csz, vp, vp]
        lib.snlm_denoise_ws.restype = ci
        lib.snlm_denoise_host.argtypes = [vp, ci, ci, ci, ci, ci, ci, cf, ci, ci, cf, cf, vp, vp]
        lib.snlm_denoise_host.restype = ci
        lib.snlm_denoise_host_many.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ci, ci, ci, ci, ci, ci, ci,
                                               cf, ci, ci, cf, cf, vp]
        lib.snlm_denoise_host_many.restype = ci
        lib.snlm_bilateral.argtypes = [vp, ci, ci, ci, cf, cf, vp, ci, vp]
        lib.snlm_bilateral.restype = ci
        lib.snlm_bf_params.argtypes = [cf, ctypes.POINTER(cf), ctypes.POINTER(cf)]
        lib.snlm_bf_params.restype = ci
        lib.snlm_denoise_bf.argtypes = [vp, ci, ci, ci, ci, ci, ci, cf, ci, ci, cf, cf, cf, cf, vp, vp]
        lib.snlm_denoise_bf.restype = ci
        lib.snlm_nlm_2d.argtypes = [vp, ci, ci, ci, ci, ci, ci, cf, ci, cf, vp, vp]
        lib.snlm_nlm_2d.restype = ci
        lib.snlm_denoise_3d.argtypes = [vp, ci, ci, ci, ci, ci, ci, cf, ci, cf, ci, vp, vp]
        lib.snlm_denoise_3d.restype = ci
        lib.snlm_nlm_1d.argtypes = [vp, ci, ci, ci, cll, cll, ci, ci, cf, ci, cf, vp, cll, cll, vp, vp, vp]
        lib.snlm_nlm_1d.restype = ci
        lib.snlm_patch_dist_1d.argtypes = [vp, ci, ci, ci, ci, ci, ci, ci, cf, vp, vp]
        lib.snlm_patch_dist_1d.restype = ci
        lib.snlm_denoise_noalloc.argtypes = [vp, ci, ci, ci, ci, ci, ci, cf, ci, ci, cf, cf, vp, vp]
        lib.snlm_denoise_noalloc.restype = ci
        lib.snlm_sure_band.argtypes = [vp, ci, ci, ci, ci, ci, ci, cf, ci, cf, ci, ci, vp, vp, vp, vp, csz, vp]
        lib.snlm_sure_band.restype = ci
        lib.snlm_sure_theta.argtypes = [dp, cf, dp]
        lib.snlm_sure_theta.restype = ci
        lib.snlm_sure_combine.argtypes = [vp, vp, cll, ctypes.c_double, ctypes.c_double, vp, vp]
        lib.snlm_sure_combine.restype = ci
        pp = ctypes.POINTER(ctypes.c_void_p)
        lib.snlm_batch_plan_create.argtypes = [ctypes.POINTER(Request), ci, ctypes.POINTER(BatchConfig), pp]
        lib.snlm_batch_plan_create.restype = ci
        lib.snlm_batch_plan_workspace_bytes.argtypes = [vp]
        lib.snlm_batch_plan_workspace_bytes.restype = csz
        lib.snlm_batch_plan_upload.argtypes = [vp, vp, csz, vp]
        lib.snlm_batch_plan_upload.restype = ci
        lib.snlm_batch_plan_launch.argtypes = [vp, vp]
        lib.snlm_batch_plan_launch.restype = ci
        lib.snlm_batch_plan_capture.argtypes = [vp, vp]
        lib.snlm_batch_plan_capture.restype = ci
        lib.snlm_batch_plan_status.argtypes = [vp, vp]
        lib.snlm_batch_plan_status_async.argtypes = [vp, vp, vp]
        lib.snlm_batch_plan_status_async.restype = ci
        lib.snlm_batch_plan_status.restype = ci
        lib.snlm_batch_plan_info.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(ci)]
        lib.snlm_batch_plan_info.restype = ci
        lib.snlm_batch_plan_destroy.argtypes = [vp]
        lib.snlm_batch_plan_destroy.restype = None
        lib.snlm_trace_enable.argtypes = [ci]
        lib.snlm_trace_enable.restype = ci
        lib.snlm_trace_read.argtypes = [ctypes.POINTER(ci), fp, ci, ctypes.POINTER(ci)]
        lib.snlm_trace_read.restype = ci
        lib.snlm_kernel_name.argtypes = [ci]
        lib.snlm_kernel_name.restype = ctypes.c_char_p
        lib.snlm_probe_peaks.argtypes = [dp, vp]
        lib.snlm_probe_peaks.restype = ci
        lib.snlm_set_option.argtypes = [ci, ctypes.c_longlong]
        lib.snlm_set_option.restype = ci
        lib.snlm_get_option.argtypes = [ci]
        lib.snlm_get_option.restype = ctypes.c_longlong
        lib.snlm_device_error.argtypes = [vp]
        lib.snlm_device_error.restype = ci
        lib.snlm_server_create.argtypes = [ctypes.POINTER(ServerConfig), pp]
        lib.snlm_server_create.restype = ci
        lib.snlm_server_submit.argtypes = [vp, ctypes.POINTER(ServeRequest), ci, ctypes.POINTER(ci)]
        lib.snlm_server_submit.restype = ci
        lib.snlm_server_drain.argtypes = [vp]
        lib.snlm_server_drain.restype = ci
        lib.snlm_server_result.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ci)]
        lib.snlm_server_result.restype = ci
        lib.snlm_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        lib.snlm_server_get_stats.restype = ci
        lib.snlm_server_clock.argtypes = [vp]
        lib.snlm_server_clock.restype = ctypes.c_double
        lib.snlm_server_destroy.argtypes = [vp]
        lib.snlm_server_destroy.restype = None
        del fp, dp
        _lib = lib
        return lib


# names declared in include/snlm.h (checked by the ABI test)
EXPORTED = [
    "snlm_status_str", "snlm_version", "snlm_default_h", "snlm_workspace_bytes", "snlm_denoise",
    "snlm_denoise_ws", "snlm_denoise_host", "snlm_denoise_host_many", "snlm_bilateral", "snlm_bf_params",
    "snlm_denoise_bf", "snlm_nlm_2d", "snlm_denoise_3d", "snlm_nlm_1d", "snlm_patch_dist_1d", "snlm_trace_enable",
    "snlm_trace_read", "snlm_kernel_name", "snlm_denoise_noalloc", "snlm_batch_plan_create",
    "snlm_batch_plan_workspace_bytes", "snlm_batch_plan_upload", "snlm_batch_plan_launch",
    "snlm_batch_plan_capture", "snlm_batch_plan_status", "snlm_batch_plan_status_async", "snlm_batch_plan_info",
    "snlm_batch_plan_destroy",
    "snlm_set_option", "snlm_get_option", "snlm_device_error", "snlm_server_create", "snlm_server_submit",
    "snlm_server_drain", "snlm_server_result", "snlm_server_get_stats", "snlm_server_clock", "snlm_server_destroy",
    "snlm_probe_peaks", "snlm_sure_band", "snlm_sure_theta", "snlm_sure_combine", "snlm_preload",
]
