"""Bounds-checking build of the library (the stand-in for a memory sanitizer): every computed index of a
staged image, of a plain-load tap and of the volume stays inside its buffer over all routes, z-runs, slab contexts,
x-vectors, frames, index rules, 16-bit storage, host input with overlapped read-back, a volume of one
voxel and a volume entirely off the detector.  Needs a GPU; builds the checking variant on first use."""
import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu


def test_no_out_of_bounds_index_anywhere(cuda_device):
    env = dict(os.environ, RCT_BUILD_VARIANT="check")
    script = Path(__file__).with_name("bounds_check_run.py")
    r = subprocess.run([sys.executable, str(script)], env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["runs"] > 200, res
    assert res["violations"] == 0, res
    assert res["worst_rel_rms"] < 1e-5, res                   # the checking build computes the same result
    assert res["control"] > 0 and res["control_after_restore"] == res["control"], res   # the checks are live
