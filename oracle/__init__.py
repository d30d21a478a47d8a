"""FP64 CPU oracle for the voxel-driven cone-beam backprojection.

TEST INFRASTRUCTURE ONLY.  This package is loaded by the test suite, by the
smoke check (to verify one small GPU run) and by the benchmark's CPU-baseline
leg.  The product path (the CUDA library and its Python binding) never
imports, links or calls it, and it imports nothing from the product path.

`rct_oracle.c` is a plain single-pass FP64 transcription of the paper's
Listing 1 (Section "Algorithm") with the readings stated in its header; this
module compiles it with gcc and exposes it through ctypes with numpy arrays.
"""
from .oracle import (build, load, backproject, backproject_voxels, round_f16, round_bf16,
                     max_threads, ORACLE_SRC, INDEX_FLOOR, INDEX_TRUNC)

__all__ = ["build", "load", "backproject", "backproject_voxels", "round_f16", "round_bf16",
           "max_threads", "ORACLE_SRC", "INDEX_FLOOR", "INDEX_TRUNC"]
