"""Build and call the FP64 C oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
ORACLE_SRC = HERE / "rct_oracle.c"
BUILD_DIR = HERE / "_build"
LIB_PATH = BUILD_DIR / "librct_oracle.so"

_lock = threading.Lock()
_lib = None


def compile_oracle(src: Path, out: Path, extra_flags=()) -> Path:
    """gcc -O2 with OpenMP; no target-specific flags, so x86_64 and aarch64 agree.

    -ffp-contract=off keeps every multiply and add separately rounded, as written.
    """
    out.parent.mkdir(parents=True, exist_ok=True)
    tmp = out.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", *extra_flags, str(src), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> Path:
    if force or not LIB_PATH.exists() or LIB_PATH.stat().st_mtime < ORACLE_SRC.stat().st_mtime:
        compile_oracle(ORACLE_SRC, LIB_PATH)
    return LIB_PATH


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    c_int, c_i64 = ctypes.c_int, ctypes.c_int64
    p_d = ctypes.POINTER(ctypes.c_double)
    p_f = ctypes.POINTER(ctypes.c_float)
    p_i64 = ctypes.POINTER(ctypes.c_int64)
    lib.rct_oracle_backproject.argtypes = [c_int, c_int, c_int, c_int, p_d, p_d, p_d, p_f,
                                           c_int, c_int, c_int, c_int, p_d]
    lib.rct_oracle_backproject.restype = c_int
    lib.rct_oracle_backproject_voxels.argtypes = [c_int, c_int, c_int, c_int, p_d, p_d, p_d, p_f,
                                                  p_i64, c_i64, c_int, c_int, p_d]
    lib.rct_oracle_backproject_voxels.restype = c_int
    lib.rct_oracle_round_f16.argtypes = [p_f, p_f, c_i64]
    lib.rct_oracle_round_f16.restype = c_int
    lib.rct_oracle_round_bf16.argtypes = [p_f, p_f, c_i64]
    lib.rct_oracle_round_bf16.restype = c_int
    lib.rct_oracle_max_threads.argtypes = []
    lib.rct_oracle_max_threads.restype = c_int
    return lib


def load(path: Path | None = None) -> ctypes.CDLL:
    """Load the oracle library (building it first if needed).  ``path`` loads a specific build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(str(path)))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(str(build())))
        return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _prep(matrices, origin, spacing, proj, W, H):
    A = np.ascontiguousarray(np.asarray(matrices, dtype=np.float64).reshape(-1, 12))
    o = np.ascontiguousarray(np.asarray(origin, dtype=np.float64).reshape(3))
    s = np.ascontiguousarray(np.asarray(spacing, dtype=np.float64).reshape(3))
    p = np.ascontiguousarray(np.asarray(proj, dtype=np.float32))
    n = A.shape[0]
    if p.size != n * W * H:
        raise ValueError(f"projections hold {p.size} values, expected {n}x{H}x{W}")
    return A, o, s, p, n


INDEX_FLOOR, INDEX_TRUNC = 0, 1


def backproject(L, W, H, matrices, origin, spacing, proj, *, z_range=None, n_threads=1,
                vol=None, lib=None, index_rule=INDEX_FLOOR) -> np.ndarray:
    """FP64 backprojection of all given views; returns (nz, L, L) float64 (accumulated into ``vol``).
    ``index_rule`` INDEX_TRUNC takes Listing 1's truncating (int) cast for the cell instead of floor."""
    lib = lib or load()
    A, o, s, p, n = _prep(matrices, origin, spacing, proj, W, H)
    z0, z1 = (0, L) if z_range is None else z_range
    if vol is None:
        vol = np.zeros((z1 - z0, L, L), dtype=np.float64)
    if vol.dtype != np.float64 or not vol.flags.c_contiguous or vol.size != (z1 - z0) * L * L:
        raise ValueError("vol must be a C-contiguous float64 array of the slab's size")
    rc = lib.rct_oracle_backproject(L, W, H, n, _ptr(A, ctypes.c_double), _ptr(o, ctypes.c_double),
                                    _ptr(s, ctypes.c_double), _ptr(p, ctypes.c_float),
                                    z0, z1, n_threads, index_rule, _ptr(vol, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"rct_oracle_backproject failed with code {rc}")
    return vol


def backproject_voxels(L, W, H, matrices, origin, spacing, proj, flat_idx, *, n_threads=1,
                       lib=None, index_rule=INDEX_FLOOR) -> np.ndarray:
    """FP64 sums for the voxels with flat indices ``flat_idx`` (z*L*L + y*L + x)."""
    lib = lib or load()
    A, o, s, p, n = _prep(matrices, origin, spacing, proj, W, H)
    idx = np.ascontiguousarray(np.asarray(flat_idx, dtype=np.int64))
    out = np.zeros(idx.shape, dtype=np.float64)
    rc = lib.rct_oracle_backproject_voxels(L, W, H, n, _ptr(A, ctypes.c_double),
                                           _ptr(o, ctypes.c_double), _ptr(s, ctypes.c_double),
                                           _ptr(p, ctypes.c_float), _ptr(idx, ctypes.c_int64),
                                           idx.size, n_threads, index_rule, _ptr(out, ctypes.c_double))
    if rc != 0:
        raise RuntimeError(f"rct_oracle_backproject_voxels failed with code {rc}")
    return out


def _round(fn, x) -> np.ndarray:
    src = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    dst = np.empty_like(src)
    rc = fn(_ptr(src, ctypes.c_float), _ptr(dst, ctypes.c_float), src.size)
    if rc != 0:
        raise RuntimeError("rounding failed")
    return dst


def round_f16(x, lib=None) -> np.ndarray:
    """Nearest IEEE binary16 value of each FP32 input (ties to even), as float32."""
    return _round((lib or load()).rct_oracle_round_f16, x)


def round_bf16(x, lib=None) -> np.ndarray:
    """Nearest bfloat16 value of each FP32 input (ties to even), as float32."""
    return _round((lib or load()).rct_oracle_round_bf16, x)


def max_threads(lib=None) -> int:
    return int((lib or load()).rct_oracle_max_threads())
