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


def test_traffic_records(tmp_path, monkeypatch):
    """Traffic per launch comes from a record in a profile summary, and counts only for the same volume size,
    storage type, tuning and kernel source."""
    for rec in bench.traffic_records():                     # every committed record is well formed
        assert rec["dtype"] in ("f32", "f16", "bf16")
        assert set(rec["tuning"]) - {"view_split"} == {"block_x", "block_y", "gather", "tex_zrun",
                                                        "views_per_pass", "xvec", "zrun"}
        assert rec["L"] in (128, 256, 512, 1024)
        # one accumulating pass: the volume read and written plus the pass's views (a capture can end with
        # some of the volume's writes still in L2; a register-capped kernel's spills can add up to its
        # algorithmic bytes again)
        algo = 2 * 4 * rec["L"] ** 3 + rec["tuning"]["views_per_pass"] * 4 * 1248 * 960
        assert 0.85 * algo < rec["bytes"] < 2.0 * algo
        assert rec["updates"] == rec["L"] ** 3 * rec["tuning"]["views_per_pass"]
        if "lsu_wavefronts" in rec:                          # 1-40 wavefronts per warp update
            assert rec["updates"] / 32 < rec["lsu_wavefronts"] < 40 * rec["updates"] / 32
        assert len(rec["kernel_source"]) == 16
    tun = {"block_x": 8, "block_y": 16, "gather": 5, "tex_zrun": 0, "views_per_pass": 24, "xvec": 1, "zrun": 8}
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"dtype": "f32", "L": 512, "tuning": tun, "kernel_source": bench.kernel_source_hash(),
           "bytes": 1269302272, "updates": 512 ** 3 * 24}
    (prof / "x.md").write_text("# summary\n\ntraffic-record: " + json.dumps(rec) + "\n")
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    for rel in bench.KERNEL_SOURCES:                        # the same kernel sources under the fake root
        (tmp_path / rel).parent.mkdir(parents=True, exist_ok=True)
        (tmp_path / rel).write_bytes((real_root / rel).read_bytes())
    got = bench.recorded_traffic("f32", tun, 512)
    assert got["bytes"] == 1269302272 and got["source"] == "x.md"
    assert bench.recorded_traffic("f32", dict(tun, view_split=1), 512)["bytes"] == 1269302272
    assert bench.recorded_traffic("f32", dict(tun, view_split=2), 512) is None
    assert bench.recorded_traffic("f32", tun, 1024) is None
    assert bench.recorded_traffic("f16", tun, 512) is None
    assert bench.recorded_traffic("f32", dict(tun, zrun=16), 512) is None
    (tmp_path / bench.KERNEL_SOURCES[0]).write_text("// changed kernel\n")
    assert bench.recorded_traffic("f32", tun, 512) is None


def _json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def test_reference_arm_line_contract():
    """`bench.py --impl reference` on a tiny workload: one JSON line with the contract's keys, the oracle's
    rate as value, cpu_baseline and e2e carrying the same value and no host-device bytes."""
    import subprocess
    r = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--workload", "tiny_L16",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1, r.stdout
    d = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "GUPS" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1 and d["vs_baseline"] is None
    assert d["value"] > 0 and d["config"]["workload"].startswith("tiny_L16")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "GUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_torchrun_prints_once():
    """Launched as two ranks (gloo on the CPU), rank 0 alone runs and prints; both ranks exit 0."""
    import socket
    import subprocess
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), str(ROOT / "bench.py"),
                        "--impl", "reference", "--workload", "tiny_L16", "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2, r.stdout


def test_wait_for_host_link_is_bounded(monkeypatch):
    """The end-to-end and served legs wait for a plain host-to-device copy at half the link's rate, in 5 s
    steps, and give up after LINK_WAIT_S; a ready link costs no wait."""
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    monkeypatch.setattr(bench, "_link_wait_spent", [0.0])
    assert bench.wait_for_host_link(lambda: 0.0, 210.0) == {"seconds": 0.0, "h2d_samples": []}
    rates = iter([2.7, 9.4, 209.9])
    got = bench.wait_for_host_link(lambda: next(rates), 1.9)
    assert got == {"seconds": 15.0, "h2d_samples": [2.7, 9.4, 209.9]}
    monkeypatch.setattr(bench, "_link_wait_spent", [0.0])
    slow = bench.wait_for_host_link(lambda: 3.0, 3.0)
    assert slow["seconds"] == bench.LINK_WAIT_S and len(slow["h2d_samples"]) == int(bench.LINK_WAIT_S / 5)
    # the waits of one run share a total bound
    rest = bench.wait_for_host_link(lambda: 3.0, 3.0)
    assert rest["seconds"] == bench.LINK_WAIT_TOTAL_S - bench.LINK_WAIT_S
    assert bench.wait_for_host_link(lambda: 3.0, 3.0)["seconds"] == 0.0
