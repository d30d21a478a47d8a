"""ctypes binding of the measurement library librct_bench.so (include/rct_bench.h).

The throughput probes measure the ceilings the benchmark reports the
backprojection against.  They are not part of the product library: only the
benchmark loads them.  A non-OK status raises ``RctError``.
"""
from __future__ import annotations

import ctypes
import threading

from . import build as _build
from .rct import RctError, STATUS_NAMES  # noqa: F401  (re-exported for callers)

_lock = threading.Lock()
_lib = None

_I = ctypes.c_int
_PD = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "rct_probe_texture": (_I, [_I, _I, ctypes.c_float, ctypes.c_float, _I, _PD]),
    "rct_probe_update_stream": (_I, [ctypes.c_size_t, _PD]),
    "rct_probe_l1_bandwidth": (_I, [_I, _PD]),
    "rct_probe_l2_sectors": (_I, [_I, _PD]),
    "rct_probe_gather_pattern": (_I, [ctypes.POINTER(ctypes.c_float), ctypes.c_float, ctypes.c_float, _I, _PD]),
}


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _build.build()
            handle = ctypes.CDLL(str(_build.BENCH_LIB))
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
        return _lib


def _check(status: int, what: str) -> None:
    if status != 0:
        raise RctError(status, what)


def rct_probe_texture(mode: int, dtype: int, stride_px: float, step_px: float, iters: int = 4096) -> float:
    r = ctypes.c_double()
    _check(lib().rct_probe_texture(mode, dtype, stride_px, step_px, iters, ctypes.byref(r)), "rct_probe_texture")
    return r.value


def rct_probe_update_stream(nbytes: int) -> float:
    r = ctypes.c_double()
    _check(lib().rct_probe_update_stream(nbytes, ctypes.byref(r)), "rct_probe_update_stream")
    return r.value


def rct_probe_l1_bandwidth(iters: int = 4096) -> float:
    r = ctypes.c_double()
    _check(lib().rct_probe_l1_bandwidth(iters, ctypes.byref(r)), "rct_probe_l1_bandwidth")
    return r.value


def rct_probe_l2_sectors(iters: int = 2048) -> float:
    r = ctypes.c_double()
    _check(lib().rct_probe_l2_sectors(iters, ctypes.byref(r)), "rct_probe_l2_sectors")
    return r.value


def rct_probe_gather_pattern(lane_uv, step_u: float, step_v: float, iters: int = 1024) -> float:
    """Cells per second of the plain-load gather with the warp footprint ``lane_uv`` (32 x 2 pixel offsets)."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(lane_uv, dtype=np.float32).reshape(64))
    r = ctypes.c_double()
    _check(lib().rct_probe_gather_pattern(a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), float(step_u),
                                          float(step_v), iters, ctypes.byref(r)), "rct_probe_gather_pattern")
    return r.value
