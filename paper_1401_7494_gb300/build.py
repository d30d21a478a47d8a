"""Compile the CUDA libraries in-tree for sm_103a (nvcc, no cmake).

Translation units are compiled in parallel into ``_build/`` next to this
file and linked into ``_build/librct.so``, the product library, and
``_build/librct_bench.so``, the throughput probes the benchmark measures its
ceilings with (``csrc/rct_probe.cu``; include/rct_bench.h).  The CUDA runtime
is linked statically, so both load on a machine without a GPU.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
# RCT_BUILD_VARIANT=check builds (and the binding loads) the bounds-checking library in its own folder
VARIANTS = {"": ("_build", []), "check": ("_build_check", ["-DRCT_CHECK_BOUNDS"])}
VARIANT = os.environ.get("RCT_BUILD_VARIANT", "")
if VARIANT not in VARIANTS:
    raise RuntimeError(f"RCT_BUILD_VARIANT={VARIANT!r}: expected one of {sorted(VARIANTS)}")
BUILD = PKG / VARIANTS[VARIANT][0]
LIB = BUILD / "librct.so"
BENCH_LIB = BUILD / "librct_bench.so"
BENCH_SOURCES = ("rct_probe.cu",)
INCLUDE = PKG.parent / "include"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not Path(exe).exists():
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return exe


def sources():
    """Translation units of the product library."""
    return sorted(p for p in CSRC.glob("*.cu") if p.name not in BENCH_SOURCES)


def bench_sources():
    return sorted(CSRC / n for n in BENCH_SOURCES)


def _deps():
    return (sources() + bench_sources() + sorted(CSRC.glob("*.h")) + sorted(CSRC.glob("*.cuh"))
            + sorted(INCLUDE.glob("*.h")))


def up_to_date() -> bool:
    if not LIB.exists() or not BENCH_LIB.exists():
        return False
    t = min(LIB.stat().st_mtime, BENCH_LIB.stat().st_mtime)
    return all(p.stat().st_mtime <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> Path:
    if not force and up_to_date():
        return LIB
    BUILD.mkdir(parents=True, exist_ok=True)
    exe = nvcc()

    def compile_one(src: Path) -> Path:
        obj = BUILD / (src.stem + ".o")
        cmd = [exe, *ARCH, *NVCC_FLAGS, *VARIANTS[VARIANT][1], *extra_flags, "-c", str(src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources() + bench_sources()))
    names = {o.stem for o in objs}
    bench_objs = [o for o in objs if o.stem in {Path(n).stem for n in BENCH_SOURCES}]
    lib_objs = [o for o in objs if o not in bench_objs]
    assert len(names) == len(objs)
    for target, parts in ((LIB, lib_objs), (BENCH_LIB, bench_objs)):
        tmp = BUILD / f"{target.stem}.{os.getpid()}.so"
        cmd = [exe, *ARCH, "-shared", "-cudart", "static", "-o", str(tmp), *map(str, parts)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link of {target.name} failed:\n{r.stderr}")
        os.replace(tmp, target)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
