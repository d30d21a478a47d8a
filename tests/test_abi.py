"""The C-ABI library: builds, loads without a GPU, exports every declared symbol; host logic (CPU)."""
import re
import subprocess
from pathlib import Path

import numpy as np
import pytest

import synth
from paper_1401_7494_gb300 import rct
from paper_1401_7494_gb300 import build as pkg_build

ROOT = Path(__file__).resolve().parents[1]


def declared_symbols(*headers):
    names = set()
    for name in headers:
        text = (ROOT / "include" / name).read_text()
        names |= set(re.findall(r"^RCT_API\s+[\w\s\*]*?\b(rct_\w+)\s*\(", text, flags=re.M))
    return names


def exported(path):
    out = subprocess.run(["nm", "-D", "--defined-only", str(path)], capture_output=True, text=True,
                         check=True).stdout
    return set(re.findall(r"\bT (rct_\w+)$", out, flags=re.M))


def test_every_header_is_covered():
    assert sorted(p.name for p in (ROOT / "include").glob("*.h")) == ["rct.h", "rct_bench.h", "rct_debug.h"]


def test_every_declared_symbol_is_exported():
    decl = declared_symbols("rct.h", "rct_debug.h")
    assert {"rct_create", "rct_backproject", "rct_set_geometry", "rct_read_volume", "rct_create_slab"} <= decl
    lib = rct.lib()
    exp = exported(pkg_build.LIB)
    assert decl <= exp, f"declared but not exported: {sorted(decl - exp)}"
    assert not {n for n in exp if n.startswith("rct_probe")}, "probes belong to the measurement library"
    for name in decl:
        assert hasattr(lib, name)
    assert set(rct.SIGNATURES) == decl, "binding and header disagree"


def test_measurement_library_exports_the_probes():
    from paper_1401_7494_gb300 import probes
    decl = declared_symbols("rct_bench.h")
    assert decl == {"rct_probe_texture", "rct_probe_update_stream", "rct_probe_l1_bandwidth", "rct_probe_l2_sectors",
                    "rct_probe_gather_pattern"}
    probes.lib()
    assert decl <= exported(pkg_build.BENCH_LIB)
    assert set(probes.SIGNATURES) == decl


def test_version_and_error_channel():
    assert rct.rct_version() >= 10000
    with pytest.raises(rct.RctError) as e:
        rct.rct_fold_geometry(0, np.zeros(12), np.zeros(3), np.ones(3))
    assert e.value.status == rct.RCT_EINVAL
    assert "L = 0" in rct.rct_last_error()


def test_fold_geometry_reproduces_projection_in_fp64():
    """(u', v', w) from the folded rows equal (u - cu w, v - cv w, w) of the original matrix."""
    w = synth.make_workload(33, n_views=7, det_w=120, det_h=90, seed=3)
    fold, shift = rct.rct_fold_geometry(w.L, w.geom.matrices, w.origin, w.spacing)
    rng = np.random.default_rng(0)
    vox = rng.integers(0, w.L, size=(50, 3)).astype(np.float64)
    cen = (w.L - 1) / 2.0
    for k in range(w.n_views):
        world = w.origin + vox * w.spacing
        u, v, ww = (w.geom.matrices[k] @ np.c_[world, np.ones(50)].T)
        up, vp, wp = fold[k] @ np.c_[vox - cen, np.ones(50)].T
        cu, cv = shift[k]
        assert np.allclose(wp, ww, rtol=1e-13)
        assert np.allclose(up, u - cu * ww, rtol=1e-12, atol=1e-9)
        assert np.allclose(vp, v - cv * ww, rtol=1e-12, atol=1e-9)
        # the shift is the pixel nearest to the projection of the volume centre
        c = w.geom.matrices[k] @ np.r_[w.origin + cen * w.spacing, 1.0]
        assert (cu, cv) == (round(c[0] / c[2]), round(c[1] / c[2]))


def test_fold_geometry_rejects_bad_input():
    m = np.zeros((1, 12))
    with pytest.raises(rct.RctError):
        rct.rct_fold_geometry(8, m, np.zeros(3), np.array([1.0, 0.0, 1.0]))
    with pytest.raises(rct.RctError):
        rct.rct_fold_geometry(8, np.full(12, np.nan), np.zeros(3), np.ones(3))


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rct.RctError):
        rct.rct_create(8, 16, 16, 4)
