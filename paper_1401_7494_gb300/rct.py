"""ctypes binding of the C ABI in include/rct.h (argument marshalling only).

Every function has the name and argument order of its C counterpart.  Device
buffers may be given as torch tensors (their ``data_ptr()`` is passed) or as
integer addresses; streams as ``torch.cuda.Stream`` objects, raw integer
handles or None (the legacy default stream).  A non-OK status raises
``RctError`` carrying the library's message.  There is no fallback: if the
compiled library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

RCT_OK, RCT_EINVAL, RCT_ENOMEM, RCT_ECUDA, RCT_ESTATE, RCT_ETIMEOUT, RCT_ENOTSUP = range(7)
RCT_PROJ_F32, RCT_PROJ_F16, RCT_PROJ_BF16 = 0, 1, 2
RCT_INTERP_SOFT, RCT_INTERP_TEX = 0, 1
RCT_FRAME_GLOBAL, RCT_FRAME_BLOCK = 0, 1
RCT_INDEX_FLOOR, RCT_INDEX_TRUNC = 0, 1
RCT_GATHER_AUTO, RCT_GATHER_LDG, RCT_GATHER_TLD4, RCT_GATHER_MIX, RCT_GATHER_QUAD, RCT_GATHER_PAIR, RCT_GATHER_DQUAD = range(7)
RCT_MAX_VIEWS_PER_PASS = 32
STATUS_NAMES = {0: "RCT_OK", 1: "RCT_EINVAL", 2: "RCT_ENOMEM", 3: "RCT_ECUDA", 4: "RCT_ESTATE",
                5: "RCT_ETIMEOUT", 6: "RCT_ENOTSUP"}


class RctError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class rct_tuning(ctypes.Structure):
    _fields_ = [("views_per_pass", ctypes.c_int), ("zrun", ctypes.c_int), ("xvec", ctypes.c_int),
                ("block_x", ctypes.c_int), ("block_y", ctypes.c_int), ("gather", ctypes.c_int),
                ("tex_zrun", ctypes.c_int), ("view_split", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D3 = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "rct_create": (_P, [_I, _I, _I, _I]),
    "rct_create_slab": (_P, [_I, _I, _I, _I, _I, _I]),
    "rct_get_slab": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rct_get_precision": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rct_destroy": (None, [_P]),
    "rct_set_geometry": (_I, [_P, _D3, _D3, _D3]),
    "rct_set_precision": (_I, [_P, _I, _I]),
    "rct_set_frame": (_I, [_P, _I]),
    "rct_get_frame": (_I, [_P, ctypes.POINTER(ctypes.c_int)]),
    "rct_set_index_rule": (_I, [_P, _I]),
    "rct_debug_bound_violations": (_I, [_P, ctypes.POINTER(ctypes.c_ulonglong)]),
    "rct_debug_lower_bound_limit": (_I, [_P, ctypes.c_longlong]),
    "rct_set_filter": (_I, [_P, ctypes.c_double, ctypes.c_double, _D3]),
    "rct_filter_projections": (_I, [_P, _P, _P, _I, _I, _I, _P]),
    "rct_get_index_rule": (_I, [_P, ctypes.POINTER(ctypes.c_int)]),
    "rct_set_geometry_rabbitct": (_I, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_float, ctypes.c_float]),
    "rct_set_tuning": (_I, [_P, ctypes.POINTER(rct_tuning)]),
    "rct_get_tuning": (_I, [_P, ctypes.POINTER(rct_tuning)]),
    "rct_reset_volume": (_I, [_P, _P]),
    "rct_backproject": (_I, [_P, _P, _I, _I, _P]),
    "rct_backproject_host": (_I, [_P, _P, _I, _I, _P]),
    "rct_backproject_host_read": (_I, [_P, _P, _I, _I, _P, _P]),
    "rct_read_volume": (_I, [_P, _P, _P]),
    "rct_write_volume": (_I, [_P, _P, _P]),
    "rct_volume_device_ptr": (_P, [_P]),
    "rct_get_shape": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rct_launch_count": (ctypes.c_int64, [_P]),
    "rct_profile_kernels": (_I, [_P, _I]),
    "rct_profile_read": (_I, [_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "rct_convert_projections": (_I, [_P, _P, ctypes.c_size_t, _I, _P]),
    "rct_fold_geometry": (_I, [_I, _I, _D3, _D3, _D3, _D3, ctypes.POINTER(_I)]),
    "rct_prepare": (_I, [_P, _I]),
    "rct_footprint_bytes": (ctypes.c_size_t, [_I, _I, _I, _I, _I, _I]),
    "rct_graph_begin": (_I, [_P]),
    "rct_graph_end": (_I, [_P, ctypes.POINTER(_P)]),
    "rct_graph_launch": (_I, [_P, _P]),
    "rct_graph_destroy": (None, [_P]),
    "rct_backproject_f16_noalloc": (_I, [_I, _I, _I, _D3, _I, _D3, _D3, _P, _P, _I, _P]),
    "rct_last_error": (ctypes.c_char_p, []),
    "rct_version": (_I, []),
}


def lib() -> ctypes.CDLL:
    """Load (building first if the sources are newer) the in-tree librct.so."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            handle = ctypes.CDLL(str(path))
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
        return _lib


def library_path() -> str:
    return str(_build.LIB)


def _check(status: int) -> None:
    if status != RCT_OK:
        raise RctError(status, lib().rct_last_error().decode(errors="replace"))


def _addr(buf) -> int | None:
    """Address of a torch tensor, numpy array or raw integer."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("buffer must be contiguous")
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return buf.ctypes.data
    raise TypeError(f"cannot take the address of {type(buf).__name__}")


_ELEM = {RCT_PROJ_F32: 4, RCT_PROJ_F16: 2, RCT_PROJ_BF16: 2}


def _torch_dtypes(code: int):
    import torch
    return {RCT_PROJ_F32: (torch.float32,), RCT_PROJ_F16: (torch.float16,),
            RCT_PROJ_BF16: (torch.bfloat16,)}[code]


def _np_dtypes(code: int):
    return {RCT_PROJ_F32: (np.float32,), RCT_PROJ_F16: (np.float16,), RCT_PROJ_BF16: ()}[code]


def _check_buffer(buf, what: str, *, code: int, min_elems: int, where: str) -> None:
    """Validate a tensor or array before its address goes to the library: its element type (the
    rct_proj_dtype ``code``), its size (at least ``min_elems`` elements) and where it lives
    (``where`` = "device": a CUDA tensor on the current device; "host": host memory; "any": either).
    Raw integer addresses cannot be checked and are passed through.  Raises ValueError."""
    if buf is None or isinstance(buf, int):
        return
    if hasattr(buf, "data_ptr") and hasattr(buf, "dtype"):
        import torch
        if buf.dtype not in _torch_dtypes(code):
            raise ValueError(f"{what}: dtype {buf.dtype} where {_torch_dtypes(code)[0]} is expected")
        if buf.is_cuda:
            if where == "host":
                raise ValueError(f"{what}: a host buffer is expected, got a tensor on {buf.device}")
            cur = torch.cuda.current_device()
            if buf.device.index != cur:
                raise ValueError(f"{what}: tensor on {buf.device} but cuda:{cur} is the current device")
        else:
            if where == "device":
                raise ValueError(f"{what}: a CUDA tensor is expected, got one on {buf.device}")
            if buf.device.type != "cpu":
                raise ValueError(f"{what}: tensors on {buf.device} cannot be passed")
        n = buf.numel()
    elif isinstance(buf, np.ndarray):
        if where == "device":
            raise ValueError(f"{what}: a CUDA tensor is expected, got a numpy array")
        if buf.dtype.type not in _np_dtypes(code) and not (code == RCT_PROJ_BF16 and buf.dtype == np.uint16):
            raise ValueError(f"{what}: dtype {buf.dtype} does not match the storage type")
        n = buf.size
    else:
        return
    if n < min_elems:
        raise ValueError(f"{what}: {n} elements, at least {min_elems} needed")


def _ctx_sizes(ctx) -> tuple[int, int, int, int, int, int]:
    """(L, det_w, det_h, planes held, proj dtype code, interp) of a context."""
    L, W, H, _ = rct_get_shape(ctx)
    _, zc = rct_get_slab(ctx)
    dt, it = rct_get_precision(ctx)
    return L, W, H, zc, dt, it


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _f64(a, n: int):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    return arr, arr.ctypes.data_as(_D3)


# ----------------------------------------------------------------------------- C names

def rct_version() -> int:
    return lib().rct_version()


def rct_last_error() -> str:
    return lib().rct_last_error().decode(errors="replace")


def rct_create(L: int, det_w: int, det_h: int, n_views: int) -> int:
    h = lib().rct_create(L, det_w, det_h, n_views)
    if not h:
        raise RctError(RCT_EINVAL, rct_last_error())
    return h


def rct_create_slab(L: int, det_w: int, det_h: int, n_views: int, z_first: int, z_count: int) -> int:
    h = lib().rct_create_slab(L, det_w, det_h, n_views, z_first, z_count)
    if not h:
        raise RctError(RCT_EINVAL, rct_last_error())
    return h


def rct_get_slab(ctx) -> tuple[int, int]:
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().rct_get_slab(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def rct_get_precision(ctx) -> tuple[int, int]:
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib().rct_get_precision(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def rct_destroy(ctx) -> None:
    if ctx:
        lib().rct_destroy(ctx)


def rct_set_geometry(ctx, matrices, origin, spacing) -> None:
    m = np.ascontiguousarray(np.asarray(matrices, dtype=np.float64).reshape(-1))
    if m.size % 12:
        raise ValueError("matrices must hold 12 values per view")
    o, po = _f64(origin, 3)
    s, ps = _f64(spacing, 3)
    _check(lib().rct_set_geometry(ctx, m.ctypes.data_as(_D3), po, ps))


def rct_set_precision(ctx, proj_dtype: int, interp: int = RCT_INTERP_SOFT) -> None:
    _check(lib().rct_set_precision(ctx, int(proj_dtype), int(interp)))


def rct_set_frame(ctx, frame: int) -> None:
    _check(lib().rct_set_frame(ctx, int(frame)))


def rct_get_frame(ctx) -> int:
    f = ctypes.c_int()
    _check(lib().rct_get_frame(ctx, ctypes.byref(f)))
    return f.value


def rct_set_filter(ctx, sdd: float, pitch: float, principal) -> None:
    pp = np.ascontiguousarray(np.asarray(principal, dtype=np.float64).reshape(-1))
    if pp.size % 2:
        raise ValueError("principal points come in (u0, v0) pairs")
    _check(lib().rct_set_filter(ctx, float(sdd), float(pitch), pp.ctypes.data_as(_D3)))


def rct_filter_projections(ctx, d_raw, d_out, out_dtype: int, first_view: int, n: int, stream=None) -> None:
    if not isinstance(d_raw, int) or not isinstance(d_out, int):
        _, W, H, _, _, _ = _ctx_sizes(ctx)
        _check_buffer(d_raw, "d_raw", code=RCT_PROJ_F32, min_elems=max(n, 0) * W * H, where="device")
        if out_dtype in _ELEM:
            _check_buffer(d_out, "d_out", code=int(out_dtype), min_elems=max(n, 0) * W * H, where="device")
    _check(lib().rct_filter_projections(ctx, _addr(d_raw), _addr(d_out), int(out_dtype), first_view, n,
                                        _stream(stream)))


def rct_debug_bound_violations(ctx) -> int:
    n = ctypes.c_ulonglong()
    _check(lib().rct_debug_bound_violations(ctx, ctypes.byref(n)))
    return n.value


def rct_debug_lower_bound_limit(ctx, staged_elems: int) -> None:
    _check(lib().rct_debug_lower_bound_limit(ctx, int(staged_elems)))


def rct_set_index_rule(ctx, rule: int) -> None:
    _check(lib().rct_set_index_rule(ctx, int(rule)))


def rct_get_index_rule(ctx) -> int:
    r = ctypes.c_int()
    _check(lib().rct_get_index_rule(ctx, ctypes.byref(r)))
    return r.value


def rct_set_geometry_rabbitct(ctx, matrices_colmajor, O: float, MM: float) -> None:
    m = np.ascontiguousarray(np.asarray(matrices_colmajor, dtype=np.float32).reshape(-1))
    if m.size % 12:
        raise ValueError("matrices must hold 12 values per view")
    _check(lib().rct_set_geometry_rabbitct(ctx, m.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                           ctypes.c_float(O), ctypes.c_float(MM)))


def rct_set_tuning(ctx, views_per_pass=0, zrun=0, xvec=0, block_x=0, block_y=0, gather=0, tex_zrun=0,
                   view_split=0) -> None:
    t = rct_tuning(views_per_pass, zrun, xvec, block_x, block_y, gather, tex_zrun, view_split)
    _check(lib().rct_set_tuning(ctx, ctypes.byref(t)))


def rct_get_tuning(ctx) -> dict:
    t = rct_tuning()
    _check(lib().rct_get_tuning(ctx, ctypes.byref(t)))
    return t.as_dict()


def rct_reset_volume(ctx, stream=None) -> None:
    _check(lib().rct_reset_volume(ctx, _stream(stream)))


def _check_proj(ctx, proj, n: int, where: str) -> None:
    if proj is None or isinstance(proj, int):
        return
    _, W, H, _, dt, _ = _ctx_sizes(ctx)
    _check_buffer(proj, "projections", code=dt, min_elems=max(n, 0) * W * H, where=where)


def _check_volume(ctx, vol, what: str, where: str = "any") -> None:
    if vol is None or isinstance(vol, int):
        return
    L, _, _, zc, _, _ = _ctx_sizes(ctx)
    _check_buffer(vol, what, code=RCT_PROJ_F32, min_elems=zc * L * L, where=where)


def rct_backproject(ctx, d_proj, first_view: int, n: int, stream=None) -> None:
    _check_proj(ctx, d_proj, n, "device")
    _check(lib().rct_backproject(ctx, _addr(d_proj), first_view, n, _stream(stream)))


def rct_backproject_host(ctx, h_proj, first_view: int, n: int, stream=None) -> None:
    _check_proj(ctx, h_proj, n, "host")
    _check(lib().rct_backproject_host(ctx, _addr(h_proj), first_view, n, _stream(stream)))


def rct_backproject_host_read(ctx, h_proj, first_view: int, n: int, dst, stream=None) -> None:
    _check_proj(ctx, h_proj, n, "host")
    _check_volume(ctx, dst, "dst")
    _check(lib().rct_backproject_host_read(ctx, _addr(h_proj), first_view, n, _addr(dst), _stream(stream)))


def rct_read_volume(ctx, dst, stream=None) -> None:
    _check_volume(ctx, dst, "dst")
    _check(lib().rct_read_volume(ctx, _addr(dst), _stream(stream)))


def rct_write_volume(ctx, src, stream=None) -> None:
    _check_volume(ctx, src, "src")
    _check(lib().rct_write_volume(ctx, _addr(src), _stream(stream)))


def rct_volume_device_ptr(ctx) -> int:
    p = lib().rct_volume_device_ptr(ctx)
    if not p:
        raise RctError(RCT_EINVAL, rct_last_error())
    return p


def rct_get_shape(ctx) -> tuple[int, int, int, int]:
    vals = [ctypes.c_int() for _ in range(4)]
    _check(lib().rct_get_shape(ctx, *[ctypes.byref(v) for v in vals]))
    return tuple(v.value for v in vals)


def rct_launch_count(ctx) -> int:
    return int(lib().rct_launch_count(ctx))


def rct_profile_kernels(ctx, enable: bool) -> None:
    _check(lib().rct_profile_kernels(ctx, 1 if enable else 0))


def rct_profile_read(ctx) -> tuple[float, int]:
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().rct_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def rct_convert_projections(d_src, d_dst, n: int, dtype: int, stream=None) -> None:
    _check_buffer(d_src, "d_src", code=RCT_PROJ_F32, min_elems=n, where="device")
    if dtype in _ELEM:
        _check_buffer(d_dst, "d_dst", code=int(dtype), min_elems=n, where="device")
    _check(lib().rct_convert_projections(_addr(d_src), _addr(d_dst), n, dtype, _stream(stream)))


def rct_prepare(ctx, host_input: bool = False) -> None:
    _check(lib().rct_prepare(ctx, 1 if host_input else 0))


def rct_footprint_bytes(L: int, det_w: int, det_h: int, proj_dtype: int, views_per_pass: int,
                        host_input: bool = False) -> int:
    return int(lib().rct_footprint_bytes(L, det_w, det_h, proj_dtype, views_per_pass, 1 if host_input else 0))


def rct_graph_begin(stream) -> None:
    _check(lib().rct_graph_begin(_stream(stream)))


def rct_graph_end(stream) -> int:
    g = ctypes.c_void_p()
    _check(lib().rct_graph_end(_stream(stream), ctypes.byref(g)))
    return g.value


def rct_graph_launch(graph, stream=None) -> None:
    _check(lib().rct_graph_launch(graph, _stream(stream)))


def rct_graph_destroy(graph) -> None:
    if graph:
        lib().rct_graph_destroy(graph)


def rct_backproject_f16_noalloc(L: int, det_w: int, det_h: int, matrices, origin, spacing, d_proj, n: int,
                                d_volume, accumulate: bool = False, stream=None) -> None:
    """Allocation-free FP16-storage backprojection into a caller-owned volume (see include/rct.h)."""
    m = np.ascontiguousarray(np.asarray(matrices, dtype=np.float64).reshape(-1))
    if m.size < 12 * n:
        raise ValueError("matrices must hold 12 values per view")
    _check_buffer(d_proj, "d_proj", code=RCT_PROJ_F32, min_elems=max(n, 0) * det_w * det_h, where="device")
    _check_buffer(d_volume, "d_volume", code=RCT_PROJ_F32, min_elems=L ** 3, where="device")
    o, po = _f64(origin, 3)
    s, ps = _f64(spacing, 3)
    _check(lib().rct_backproject_f16_noalloc(L, det_w, det_h, m.ctypes.data_as(_D3), n, po, ps, _addr(d_proj),
                                             _addr(d_volume), 1 if accumulate else 0, _stream(stream)))


def rct_fold_geometry(L: int, matrices, origin, spacing):
    """Host-only FP64 fold; returns (fold (n, 3, 4) float64, shift (n, 2) int32)."""
    m = np.ascontiguousarray(np.asarray(matrices, dtype=np.float64).reshape(-1))
    n = m.size // 12
    o, po = _f64(origin, 3)
    s, ps = _f64(spacing, 3)
    fold = np.zeros(12 * n, dtype=np.float64)
    shift = np.zeros(2 * n, dtype=np.int32)
    _check(lib().rct_fold_geometry(L, n, m.ctypes.data_as(_D3), po, ps, fold.ctypes.data_as(_D3),
                                   shift.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return fold.reshape(n, 3, 4), shift.reshape(n, 2)


# ----------------------------------------------------------------------------- convenience

@dataclass
class Backprojector:
    """Owns one context: an L^3 FP32 volume on the current device and a scan geometry.  With
    ``z_range=(z_first, z_count)`` the context holds only those z planes (rct_create_slab)."""
    L: int
    det_w: int
    det_h: int
    n_views: int
    z_range: tuple | None = None

    def __post_init__(self):
        if self.z_range is None:
            self.ctx = rct_create(self.L, self.det_w, self.det_h, self.n_views)
        else:
            self.ctx = rct_create_slab(self.L, self.det_w, self.det_h, self.n_views, *self.z_range)

    def close(self):
        if getattr(self, "ctx", None):
            rct_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, matrices, origin, spacing):
        rct_set_geometry(self.ctx, matrices, origin, spacing)
        return self

    def set_precision(self, proj_dtype=RCT_PROJ_F32, interp=RCT_INTERP_SOFT):
        rct_set_precision(self.ctx, proj_dtype, interp)
        return self

    def set_frame(self, frame=RCT_FRAME_GLOBAL):
        rct_set_frame(self.ctx, frame)
        return self

    def set_index_rule(self, rule=RCT_INDEX_FLOOR):
        rct_set_index_rule(self.ctx, rule)
        return self

    def set_filter(self, sdd, pitch, principal):
        rct_set_filter(self.ctx, sdd, pitch, principal)
        return self

    def filter(self, d_raw, d_out, out_dtype=RCT_PROJ_F32, first_view=0, n=None, stream=None):
        if n is None:
            n = int(d_raw.shape[0])
        rct_filter_projections(self.ctx, d_raw, d_out, out_dtype, first_view, n, stream)

    def set_tuning(self, **kw):
        rct_set_tuning(self.ctx, **kw)
        return self

    def tuning(self) -> dict:
        return rct_get_tuning(self.ctx)

    def reset(self, stream=None):
        rct_reset_volume(self.ctx, stream)

    def backproject(self, d_proj, first_view=0, n=None, stream=None):
        if n is None:
            n = int(d_proj.shape[0])
        rct_backproject(self.ctx, d_proj, first_view, n, stream)

    def backproject_host(self, h_proj, first_view=0, n=None, stream=None):
        if n is None:
            n = int(h_proj.shape[0])
        rct_backproject_host(self.ctx, h_proj, first_view, n, stream)

    def backproject_host_read(self, h_proj, dst, first_view=0, n=None, stream=None):
        if n is None:
            n = int(h_proj.shape[0])
        rct_backproject_host_read(self.ctx, h_proj, first_view, n, dst, stream)

    def read_volume(self, dst, stream=None):
        rct_read_volume(self.ctx, dst, stream)
        return dst

    def write_volume(self, src, stream=None):
        rct_write_volume(self.ctx, src, stream)

    def volume_ptr(self) -> int:
        return rct_volume_device_ptr(self.ctx)

    @property
    def launches(self) -> int:
        return rct_launch_count(self.ctx)
