"""GB300 (sm_103a) voxel-driven cone-beam backprojection behind a small C ABI.

The compute path is the CUDA library built from ``csrc/`` (``librct.so``);
``rct`` is its ctypes binding (argument marshalling only).  PyTorch is used
by callers for device memory and streams only.
"""
from . import rct
from .rct import *  # noqa: F401,F403  (the C-ABI names)

__all__ = [n for n in dir(rct) if n.startswith(("rct_", "RCT_"))] + ["Backprojector", "RctError", "rct"]
