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
LIB_PATH = os.path.join(_PKG, "libsnlm.so")

_lock = threading.Lock()
_lib = None


class LibraryMissing(RuntimeError):
    pass


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
        lib.snlm_nlm_1d.argtypes = [vp, ci, ci, ci, cll, cll, ci, ci, cf, ci, cf, vp, cll, cll, vp, vp, vp]
        lib.snlm_nlm_1d.restype = ci
        lib.snlm_patch_dist_1d.argtypes = [vp, ci, ci, ci, ci, ci, ci, ci, cf, vp, vp]
        lib.snlm_patch_dist_1d.restype = ci
        lib.snlm_denoise_noalloc.argtypes = [vp, ci, ci, ci, ci, ci, ci, cf, ci, ci, cf, cf, vp, vp]
        lib.snlm_denoise_noalloc.restype = ci
        lib.snlm_trace_enable.argtypes = [ci]
        lib.snlm_trace_enable.restype = ci
        lib.snlm_trace_read.argtypes = [ctypes.POINTER(ci), fp, ci, ctypes.POINTER(ci)]
        lib.snlm_trace_read.restype = ci
        lib.snlm_kernel_name.argtypes = [ci]
        lib.snlm_kernel_name.restype = ctypes.c_char_p
        del fp, dp
        _lib = lib
        return lib


# names declared in include/snlm.h (checked by the ABI test)
EXPORTED = [
    "snlm_status_str", "snlm_version", "snlm_default_h", "snlm_workspace_bytes", "snlm_denoise",
    "snlm_denoise_ws", "snlm_denoise_host", "snlm_nlm_1d", "snlm_patch_dist_1d", "snlm_trace_enable",
    "snlm_trace_read", "snlm_kernel_name", "snlm_denoise_noalloc",
]
