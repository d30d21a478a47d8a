"""Host-side pieces of bench.py that need no GPU: the live-warp estimate behind the texture roofline and the
shape of the DRAM-traffic table."""
import json
import sys
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import bench  # noqa: E402
import synth  # noqa: E402


def _exhaustive_live_fraction(w, bx, by, xv, R, views):
    """Every warp of the launch (32 consecutive threads of a bx x by block, x fastest, xv voxels per
    thread, a z-run of R) against every view: live when some voxel's floor cell has a tap on the detector."""
    L, W, H = w.L, w.geom.det_w, w.geom.det_h
    live = total = 0
    for gy in range(-(-L // by)):
        for gx in range(-(-L // (bx * xv))):
            for warp in range(bx * by // 32):
                for z0 in range(0, L, R):
                    pts = []
                    for lane in range(32):
                        t = warp * 32 + lane
                        x0, y = (gx * bx + t % bx) * xv, gy * by + t // bx
                        for dx in range(xv):
                            for z in range(z0, min(z0 + R, L)):
                                if x0 + dx < L and y < L:
                                    pts.append((x0 + dx, y, z))
                    if not pts:
                        continue
                    P = np.array([[w.origin[0] + x * w.spacing[0], w.origin[1] + y * w.spacing[1],
                                   w.origin[2] + z * w.spacing[2], 1.0] for x, y, z in pts])
                    for k in views:
                        u, v, ww = (P @ np.asarray(w.geom.matrices[k], dtype=np.float64).reshape(3, 4).T).T
                        i0, j0 = np.floor(u / ww), np.floor(v / ww)
                        on = (i0 >= -1) & (i0 <= W - 1) & (j0 >= -1) & (j0 <= H - 1)
                        live += bool(on.any())
                        total += 1
    return live / total


def test_live_warp_fraction_matches_exhaustive_count():
    # 64^3 with the benchmark's field of view: about 30 % of (warp, view) pairs miss the detector
    w = synth.make_workload(64, n_views=6, det_w=64, det_h=40, seed=77)
    for bx, by, xv, R in ((8, 16, 1, 8), (16, 8, 2, 4)):
        exact = _exhaustive_live_fraction(w, bx, by, xv, R, range(w.n_views))
        assert 0.5 < exact < 0.85, exact
        est = bench.live_warp_fraction(w, dict(block_x=bx, block_y=by, xvec=xv, zrun=R), n_warps=4000,
                                       n_views=w.n_views, seed=3)
        assert abs(est - exact) < 0.03, (bx, by, xv, R, est, exact)   # about 3 sampling standard deviations


def test_traffic_table_keys():
    for key, val in bench.TRAFFIC.items():
        dtype, tun = key.split(" ", 1)
        assert dtype in ("f32", "f16", "bf16")
        t = json.loads(tun)
        assert json.dumps(t, sort_keys=True) == tun          # looked up with sort_keys=True
        assert set(t) == {"block_x", "block_y", "gather", "tex_zrun", "views_per_pass", "xvec", "zrun"}
        assert 1e9 < val < 2e9                                # one accumulating pass at 512^3: ~1.1-1.3 GB
