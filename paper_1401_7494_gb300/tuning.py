"""Kernel tuning table: (views per pass K, z-run, x-vector, block shape, gather) per workload.

``lookup`` returns the launch configuration for an (L, storage dtype,
interpolation[, coordinate frame]) key: the autotuner's cached winner when the
cache holds one for this GPU (a block-frame key falls back to the global-frame
entry), else the built-in default.  The cache is a JSON file
(``tuning_cache.json`` next to this module) written by ``autotune.py``.
"""
from __future__ import annotations

import json
import os
from pathlib import Path

from . import rct

CACHE = Path(os.environ.get("RCT_TUNING_CACHE", Path(__file__).resolve().parent / "tuning_cache.json"))

DEFAULT = dict(views_per_pass=16, zrun=4, xvec=1, block_x=32, block_y=8, gather=rct.RCT_GATHER_TLD4, tex_zrun=0)


def _key(L: int, dtype: str, interp: str, frame: str = "global") -> str:
    return f"L{L}/{dtype}/{interp}" + ("/block" if frame == "block" else "")


def _gpu_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name(0)
    except Exception:
        pass
    return "any"


def load_cache(path: Path = CACHE) -> dict:
    try:
        return json.loads(Path(path).read_text())
    except (OSError, ValueError):
        return {}


def lookup(L: int, dtype: str = "f32", interp: str = "soft", gpu: str | None = None, path: Path = CACHE,
           frame: str = "global") -> dict:
    cache = load_cache(path)
    entries = cache.get(gpu or _gpu_name(), {}) or cache.get("any", {})
    hit = entries.get(_key(L, dtype, interp, frame)) or entries.get(_key(L, dtype, interp))
    if hit:
        return dict(hit["tuning"])
    t = dict(DEFAULT)
    if L % t["xvec"]:
        t["xvec"] = 1
    return t


def store(L: int, dtype: str, interp: str, tuning: dict, gups: float, gpu: str | None = None,
          path: Path = CACHE, extra: dict | None = None, frame: str = "global") -> None:
    cache = load_cache(path)
    entries = cache.setdefault(gpu or _gpu_name(), {})
    rec = {"tuning": dict(tuning), "gups": gups}
    if extra:
        rec.update(extra)
    entries[_key(L, dtype, interp, frame)] = rec
    tmp = Path(str(path) + f".{os.getpid()}.tmp")
    tmp.write_text(json.dumps(cache, indent=1, sort_keys=True))
    os.replace(tmp, path)
