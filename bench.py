#!/usr/bin/env python
"""Benchmark of the GB300 voxel-driven backprojection (GUPS = voxel updates per second).

One step = one full reconstruction of the workload: zero the L^3 volume and
backproject every view (all steps of the hot path: the FP64 geometry fold is
done once at set-up, projection staging and the backprojection passes run in
the step).  Default workload: L = 512, 496 views of 1248 x 960 FP32
projections (the RabbitCT problem size), seeded synthetic ellipsoid phantom.
Inputs (2.4 GB of projections, a 512 MB volume) are larger than the L2, so no
flush is needed between steps.

Prints ONE JSON line on rank 0.  ``--impl reference`` times the FP64 oracle on
the host cores instead (bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

METRIC = "GUPS (voxel updates/s) at 512^3 x 496, FP32 projections"
METRIC_BY_DTYPE = {"f32": METRIC, "f16": METRIC.replace("FP32", "FP16"), "bf16": METRIC.replace("FP32", "BF16")}
UNIT = "GUPS"

# DRAM bytes (read + write) of one accumulating backprojection pass come from the ncu summaries under
# profiles/: each capture that measured them carries one line
#   traffic-record: {"dtype": ..., "tuning": {...}, "kernel_source": <sha256 prefix>, "bytes": ...}
# and a record counts only for the same storage type, the same tuning and the same kernel source (the
# hash of the kernel's header files), so a changed kernel or tuning reports traffic as null.
KERNEL_SOURCES = ("paper_1401_7494_gb300/csrc/rct_bp_kernel.cuh", "paper_1401_7494_gb300/csrc/rct_internal.h")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        h.update((ROOT / rel).read_bytes())
    return h.hexdigest()[:16]


def traffic_records() -> list:
    out = []
    for md in sorted((ROOT / "profiles").glob("*.md")):
        for line in md.read_text().splitlines():
            if line.startswith("traffic-record:"):
                rec = json.loads(line.split(":", 1)[1])
                rec["source"] = md.name
                out.append(rec)
    return out


def recorded_traffic(dtype: str, tun: dict, L: int):
    """The traffic record (ncu counters of one accumulating launch: ``bytes`` = DRAM read + write, optionally
    ``lsu_wavefronts`` and the launch's voxel ``updates``) for this volume size, storage type, tuning and kernel
    source, with its summary file under ``source``; None where no capture matches."""
    src = kernel_source_hash()
    plain = lambda t: {k: v for k, v in t.items() if not (k == "view_split" and v == 1)}   # 1 = no split
    for rec in traffic_records():
        if (rec.get("dtype") == dtype and plain(rec.get("tuning", {})) == plain(tun)
                and rec.get("kernel_source") == src and rec.get("L") == L):
            return rec
    return None


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="fp32_L512")
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16"], default="f32",
                    help="storage type of the projections for the timed step (FP32 is the headline)")
    ap.add_argument("--tuning", default=None,
                    help="JSON object of rct_tuning fields that override the tuning cache for the timed step")
    ap.add_argument("--no-variants", action="store_true", help="skip the precision variants")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving run")
    ap.add_argument("--no-k-sweep", action="store_true", help="skip the views-per-pass sweep at L=1024")
    ap.add_argument("--no-prefilter", action="store_true", help="skip the device pre-processing leg")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--out", default=None, help="also write the JSON line to this file")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed plumbing

class Dist:
    """Replica bookkeeping for N > 1: every rank reconstructs its own volume on its own GPU (the
    voxels are independent, so no data-path collective exists); ranks only meet at barriers and to
    take the max of the timed region and the sum of the work done."""

    def __init__(self, want: int, backend: str | None = None):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        self.device = "cpu"
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = backend or ("nccl" if torch.cuda.is_available() else "gloo")
            self.device = f"cuda:{self.local}" if backend == "nccl" else "cpu"
            dist.init_process_group(backend)
            self.pg = dist
        if want != self.world and self.rank == 0:
            print(f"note: --gpus {want} but WORLD_SIZE={self.world}", file=sys.stderr)

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def _reduce(self, x: float, op) -> float:
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.pg.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, self.pg.ReduceOp.MAX) if self.pg else x

    def sum(self, x: float) -> float:
        return self._reduce(x, self.pg.ReduceOp.SUM) if self.pg else x

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        for line in Path(self.file.name).read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


def workload_config(name: str, w, dtype: str = "f32") -> dict:
    return {"workload": f"{name}: L={w.L}^3 volume, {w.n_views} views of {w.geom.det_w}x{w.geom.det_h} "
                        f"{dtype.upper()} projections, seeded ellipsoid phantom",
            "L": w.L, "n_views": w.n_views, "det": [w.geom.det_w, w.geom.det_h], "seed": w.seed}


# ----------------------------------------------------------------------------- CPU oracle timing

def oracle_rate(w, host_proj, target_s: float, max_planes: int | None = None):
    """Time the FP64 oracle on a slab of z-planes x all views; returns (GUPS, cores, sample text)."""
    import oracle
    threads = oracle.max_threads()
    L = w.L
    z0 = L // 2
    # calibrate on one plane per thread, then size the sample to about target_s seconds
    cal = max(1, min(L, threads))
    t = time.perf_counter()
    oracle.backproject(L, w.geom.det_w, w.geom.det_h, w.geom.matrices, w.origin, w.spacing, host_proj,
                       z_range=(z0 - cal // 2, z0 - cal // 2 + cal), n_threads=threads)
    one = max(time.perf_counter() - t, 1e-6) / cal
    planes = int(max(1, min(L, target_s / one)))
    if max_planes:
        planes = min(planes, max_planes)
    za = max(0, min(L - planes, z0 - planes // 2))
    t = time.perf_counter()
    oracle.backproject(L, w.geom.det_w, w.geom.det_h, w.geom.matrices, w.origin, w.spacing, host_proj,
                       z_range=(za, za + planes), n_threads=threads)
    dt = time.perf_counter() - t
    updates = planes * L * L * w.n_views
    sample = (f"{planes} of {L} z-planes x {w.n_views} views ({updates:.3e} updates, {dt:.1f} s, "
              f"FP64 oracle, OpenMP over planes)")
    return updates / dt / 1e9, threads, sample


def oracle_rate_one_core(w, host_proj, planes: int = 1):
    """The same oracle on one thread over `planes` middle z-planes x all views; returns (GUPS, sample text)."""
    import oracle
    z0 = w.L // 2
    t = time.perf_counter()
    oracle.backproject(w.L, w.geom.det_w, w.geom.det_h, w.geom.matrices, w.origin, w.spacing, host_proj,
                       z_range=(z0, z0 + planes), n_threads=1)
    dt = time.perf_counter() - t
    updates = planes * w.L * w.L * w.n_views
    return updates / dt / 1e9, f"{planes} z-plane(s) x {w.n_views} views on 1 thread ({dt:.1f} s)"


# ----------------------------------------------------------------------------- our arm

def measure_variant(w, proj_dev, dtype: str, interp: str, steps: int, warmup: int, stream, check_idx=None,
                    host=None, frame: str = "global", trunc: bool = False):
    """GUPS (and, when check_idx is given, error vs the oracle on sampled voxels) for one precision variant."""
    import torch
    from paper_1401_7494_gb300 import rct, tuning
    codes = {"f32": rct.RCT_PROJ_F32, "f16": rct.RCT_PROJ_F16, "bf16": rct.RCT_PROJ_BF16}
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    interp_code = rct.RCT_INTERP_SOFT if interp == "soft" else rct.RCT_INTERP_TEX
    data = proj_dev
    if dtype != "f32":
        data = torch.empty(proj_dev.shape, dtype=tdt, device=proj_dev.device)
        rct.rct_convert_projections(proj_dev, data, proj_dev.numel(), codes[dtype], stream)
    tun = tuning.lookup(w.L, dtype, interp, frame=frame)
    out = {"tuning": tun, "frame": frame, "index_rule": "trunc" if trunc else "floor"}
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_precision(codes[dtype], interp_code)
        bp.set_frame(rct.RCT_FRAME_BLOCK if frame == "block" else rct.RCT_FRAME_GLOBAL)
        bp.set_index_rule(rct.RCT_INDEX_TRUNC if trunc else rct.RCT_INDEX_FLOOR)
        bp.set_tuning(**tun)
        for _ in range(warmup):
            bp.reset(stream)
            bp.backproject(data, 0, w.n_views, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            bp.reset(stream)
            bp.backproject(data, 0, w.n_views, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out["gups"] = w.updates / (ms / 1e3) / 1e9
        out["ms_per_step"] = ms
        if check_idx is not None:
            import oracle
            vol = torch.empty((w.L,) * 3, dtype=torch.float32, device=proj_dev.device)
            bp.read_volume(vol, stream)
            torch.cuda.synchronize()
            got = vol.view(-1)[torch.from_numpy(check_idx).to(vol.device)].cpu().numpy().astype(np.float64)
            ref = oracle.backproject_voxels(w.L, w.geom.det_w, w.geom.det_h, w.geom.matrices, w.origin, w.spacing,
                                            host, check_idx, n_threads=oracle.max_threads(),
                                            index_rule=oracle.INDEX_TRUNC if trunc else oracle.INDEX_FLOOR)
            out["rel_rms_vs_fp64_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
            out["max_abs_vs_fp64_oracle"] = float(np.abs(got - ref).max() / np.abs(ref).max())
    del data
    return out


def prefilter_leg(workload: str, dev, stream, peaks: dict, bp_ms: float) -> dict:
    """Cosine weighting + ramp filtering of the workload's raw line integrals on the device
    (rct_filter_projections), timed with CUDA events, FP32 in place and fused FP16 output."""
    import torch
    import synth
    from paper_1401_7494_gb300 import rct
    w = synth.workloads.named(workload)
    raw = synth.make_projections(w.geom, w.phantom, device=dev, weighted=False, filtered=False)
    work = torch.empty_like(raw)
    out16 = torch.empty(raw.shape, dtype=torch.float16, device=dev)
    out = {"views": w.n_views, "det": [w.geom.det_w, w.geom.det_h]}
    with rct.Backprojector(16, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_filter(w.geom.sdd, w.geom.pitch, w.geom.principal)
        for name, dst, dt, per_px in [("f32", work, rct.RCT_PROJ_F32, 8), ("f16", out16, rct.RCT_PROJ_F16, 6)]:
            for _ in range(2):
                work.copy_(raw)
                bp.filter(work, dst, dt, 0, w.n_views, stream)
            torch.cuda.synchronize()
            reps, ms = 3, 0.0
            for _ in range(reps):
                work.copy_(raw)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                bp.filter(work, dst, dt, 0, w.n_views, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1) / reps
            px = w.geom.det_w * w.geom.det_h * w.n_views
            out[name] = {"ms_per_step": round(ms, 3), "views_per_s": round(w.n_views / (ms / 1e3), 1),
                         "hbm_gbs": round(px * per_px / (ms / 1e3) / 1e9, 1),
                         "hbm_frac": round(px * per_px / (ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0), 3)}
    out["pipeline_gups_f32"] = round(w.updates / ((out["f32"]["ms_per_step"] + bp_ms) / 1e3) / 1e9, 1)
    out["note"] = ("raw line integrals -> cosine weight -> Shepp-Logan ramp filter (FFT of length 4096 per row pair "
                   "in shared memory); hbm_gbs counts one FP32 read and one write per pixel; pipeline_gups_f32 = "
                   "updates / (filter + backprojection step)")
    del raw, work, out16
    return out


def convert_leg(proj, stream, peaks: dict) -> dict:
    """Narrowing of the whole projection stack to FP16 / BF16 (rct_convert_projections, one launch), timed
    with CUDA events: 4 B read + 2 B written per pixel against the measured HBM copy rate."""
    import torch
    from paper_1401_7494_gb300 import rct
    out = {}
    n = proj.numel()
    for name, tdt, code in [("f16", torch.float16, rct.RCT_PROJ_F16), ("bf16", torch.bfloat16, rct.RCT_PROJ_BF16)]:
        dst = torch.empty(proj.shape, dtype=tdt, device=proj.device)
        rct.rct_convert_projections(proj, dst, n, code, stream)
        torch.cuda.synchronize()
        reps, ms = 5, 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rct.rct_convert_projections(proj, dst, n, code, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1) / reps
        gbs = n * 6 / (ms / 1e3) / 1e9
        out[name] = {"ms": round(ms, 3), "hbm_gbs": round(gbs, 1),
                     "hbm_frac": round(gbs / peaks.get("hbm_gbs", 6800.0), 3)}
        del dst
    out["note"] = (f"{n} pixels per launch (the whole stack), 6 B of HBM traffic per pixel; peak "
                   + ("measured (MEASURED_PEAKS.json)" if "hbm_gbs" in peaks else "fallback"))
    return out


def live_warp_fraction(w, tun: dict, n_warps: int = 3000, n_views: int = 24, seed: int = 5) -> float:
    """Fraction of (warp, view) pairs the kernel's clip test keeps, estimated on sampled warps from the
    geometry (FP64): a warp of 32 consecutive threads covers XV x-voxels per thread, its threads'
    (x, y) positions and a z-run of R; it fetches for a view when some voxel's floor cell has a tap on the
    detector.  The rest of the updates issue no gather."""
    rng = np.random.default_rng(seed)
    L, bx, by, xv, R = w.L, tun["block_x"], tun["block_y"], tun["xvec"], tun["zrun"]
    lane = np.arange(32)
    views = rng.choice(w.n_views, size=min(n_views, w.n_views), replace=False)
    live = 0
    total = 0
    for _ in range(n_warps):
        # a random block, warp and z-run
        gx, gy = rng.integers(0, -(-L // (bx * xv))), rng.integers(0, -(-L // by))
        warp = rng.integers(0, (bx * by) // 32)
        t = warp * 32 + lane
        x = (gx * bx + t % bx) * xv
        y = gy * by + t // bx
        z0 = rng.integers(0, -(-L // R)) * R
        X = (x[:, None] + np.arange(xv)[None, :]).reshape(-1)
        Y = np.repeat(y, xv)
        P = np.array([[w.origin[0] + xx * w.spacing[0], w.origin[1] + yy * w.spacing[1],
                       w.origin[2] + zz * w.spacing[2], 1.0]
                      for xx, yy in zip(X, Y) if xx < L and yy < L for zz in range(z0, min(z0 + R, L))])
        if P.size == 0:
            continue
        for k in views:
            uvw = P @ w.geom.matrices[k].T
            i0 = np.floor(uvw[:, 0] / uvw[:, 2])
            j0 = np.floor(uvw[:, 1] / uvw[:, 2])
            on = (i0 >= -1) & (i0 <= w.geom.det_w - 1) & (j0 >= -1) & (j0 <= w.geom.det_h - 1)
            live += bool(on.any())
            total += 1
    return live / max(total, 1)


def warp_footprints(w, tun: dict, n_views: int = 8) -> list:
    """Projected lane offsets of one warp of the kernel's block (the 32 threads with the lowest ids of a block at
    the volume centre, its first z-run voxel), for n_views views spread over the scan: (32 x 2 offsets in pixels
    from lane 0, the step of lane 0 to the next voxel of the run), from the geometry in FP64."""
    L, bx, xv = w.L, tun["block_x"], tun["xvec"]
    lane = np.arange(32)
    x = (lane % bx) * xv + (L // 2 // (bx * xv)) * bx * xv
    y = lane // bx + L // 2
    zc = L // 2
    out = []
    for k in np.linspace(0, w.n_views - 1, n_views).round().astype(int):
        def uv(z):
            X = np.stack([w.origin[0] + x * w.spacing[0], w.origin[1] + y * w.spacing[1],
                          np.full(32, w.origin[2] + z * w.spacing[2]), np.ones(32)], axis=1)
            q = X @ w.geom.matrices[k].T
            return q[:, 0] / q[:, 2], q[:, 1] / q[:, 2]
        u0, v0 = uv(zc)
        u1, v1 = uv(zc + 1)
        off = np.stack([u0 - u0[0], v0 - v0[0]], axis=1)
        out.append((off, float(u1[0] - u0[0]), float(v1[0] - v0[0])))
    return out


def pattern_ceiling(w, tun: dict) -> float | None:
    """Mean over the footprints of warp_footprints of the plain-load gather's measured rate (cells per second)
    for that footprint, or None where a footprint exceeds the probe's limits."""
    from paper_1401_7494_gb300 import probes, rct
    rates = []
    for off, su, sv in warp_footprints(w, tun):
        try:
            rates.append(probes.rct_probe_gather_pattern(off, su, sv, 1024))
        except rct.RctError:
            return None
    return float(np.mean(rates)) if rates else None


def k_sweep(dev, stream, peaks: dict) -> dict:
    """Views per pass K against the volume stream at L = 1024 x 496: the volume is read and written once per
    pass (8/K bytes of HBM per voxel update), so small K is HBM-bound and large K fetch-bound."""
    import torch
    import synth
    from paper_1401_7494_gb300 import rct, tuning
    w = synth.workloads.named("fp32_L1024")
    proj = w.projections(device=dev)
    base = tuning.lookup(w.L, "f32", "soft")
    rows = []
    vol_bytes = 4 * w.L ** 3
    img_bytes = 4 * w.geom.det_w * w.geom.det_h
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
        for K in (1, 4, 8, 16, 24, 32):
            bp.set_tuning(**dict(base, views_per_pass=K))
            bp.reset(stream)
            bp.backproject(proj, 0, w.n_views, stream)
            torch.cuda.synchronize()
            steps = 1 if K == 1 else 2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                bp.reset(stream)
                bp.backproject(proj, 0, w.n_views, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3 / steps
            passes = -(-w.n_views // K)
            hbm_bytes = vol_bytes * (1 + 2 * (passes - 1)) + img_bytes * w.n_views
            rows.append({"K": K, "gups": round(w.updates / sec / 1e9, 1), "s_per_step": round(sec, 4),
                         "hbm_gbs": round(hbm_bytes / sec / 1e9, 1), "hbm_frac": round(hbm_bytes / sec / 1e9 / hbm_peak, 3)})
    del proj
    return {"workload": "fp32_L1024: 1024^3 x 496 views of 1248x960", "tuning": base, "rows": rows,
            "note": "algorithmic HBM bytes per step: volume written by the first pass, read and written by the others, "
                    "each view read once"}


# Host-to-device plain-copy rate (GB/s) taken as a ready host link before the end-to-end timed region: half
# of the 210 GB/s these hosts sustain from page-locked memory; the wait for it is bounded.
LINK_READY_GBS = 100.0
LINK_WAIT_S = 90.0
LINK_WAIT_TOTAL_S = 150.0      # over the whole run (the end-to-end leg and the three served modes)
_link_wait_spent = [0.0]

def wait_for_host_link(h2d_gbs, first: float) -> dict:
    """Wait, up to LINK_WAIT_S in 5 s steps, until h2d_gbs() (the rate of a plain host-to-device copy, GB/s;
    ``first`` is the rate already measured) reaches LINK_READY_GBS.  Returns the wait and the rates seen."""
    out = {"seconds": 0.0, "h2d_samples": []}
    rate = first
    limit = min(LINK_WAIT_S, LINK_WAIT_TOTAL_S - _link_wait_spent[0])
    while rate < LINK_READY_GBS and out["seconds"] < limit:
        time.sleep(5.0)
        out["seconds"] += 5.0
        rate = h2d_gbs()
        out["h2d_samples"].append(round(rate, 1))
    _link_wait_spent[0] += out["seconds"]
    return out


VM_EVENTS = ("pgmigrate_success", "compact_migrate_scanned", "compact_free_scanned", "compact_isolated",
             "compact_stall", "compact_daemon_wake", "thp_collapse_alloc", "thp_fault_alloc", "thp_fault_fallback")


def vm_events() -> dict:
    """The host's page-migration and compaction event counters (/proc/vmstat; empty where unreadable)."""
    try:
        text = Path("/proc/vmstat").read_text()
    except OSError:
        return {}
    out = {}
    for line in text.splitlines():
        k, _, v = line.partition(" ")
        if k in VM_EVENTS:
            out[k] = int(v)
    return out


def run_ours(args, dist: Dist) -> dict | None:
    import torch
    import synth
    from paper_1401_7494_gb300 import probes, rct, tuning

    if dist.world > 1:
        # the per-GPU characterisation legs (variants, pre-filter, K sweep, serving, CPU baseline) describe one
        # GPU and would hold every replica's GPU while rank 0 runs them: at N > 1 only the step and e2e run
        args.no_variants = args.no_prefilter = args.no_k_sweep = args.no_serve = args.no_cpu_baseline = True
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    stream = torch.cuda.current_stream()
    peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text()) if (ROOT / "MEASURED_PEAKS.json").exists() else {}

    w = synth.workloads.named(args.workload)
    proj = w.projections(device=dev)                    # FP32, device resident
    codes = {"f32": rct.RCT_PROJ_F32, "f16": rct.RCT_PROJ_F16, "bf16": rct.RCT_PROJ_BF16}
    data = proj                                         # the timed step's projections, in the storage type
    if args.dtype != "f32":
        data = torch.empty(proj.shape, dtype={"f16": torch.float16, "bf16": torch.bfloat16}[args.dtype], device=dev)
        rct.rct_convert_projections(proj, data, proj.numel(), codes[args.dtype], stream)
    torch.cuda.synchronize()
    host_bufs = None
    if not args.no_e2e:
        # The end-to-end leg's page-locked host buffers, backed by aligned huge pages (hostmem: copies run at the
        # link rate without the stalls that base-page pinned buffers show on hosts whose memory has been
        # churned).  They are allocated here, before the timed step, so that any memory compaction the huge-page
        # requests set off on the host has the step's duration to settle before the end-to-end copies are timed;
        # they are locked and registered only then (hostmem.finish), after one more try for huge pages where
        # the first attempt got base pages.
        from paper_1401_7494_gb300 import hostmem
        host_bufs = (hostmem.pinned_empty(data.shape, data.dtype, register=False),
                     hostmem.pinned_empty((w.L,) * 3, torch.float32, register=False))
        huge_at_allocation = {"projections": round(hostmem.huge_fraction(host_bufs[0]), 3),
                              "volume": round(hostmem.huge_fraction(host_bufs[1]), 3)}
        host_bufs[0].copy_(data)
    tun = tuning.lookup(w.L, args.dtype, "soft")
    if args.tuning:
        tun = dict(tun, **json.loads(args.tuning))
    bp = rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views)
    bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_precision(codes[args.dtype], rct.RCT_INTERP_SOFT)
    bp.set_tuning(**tun)

    def step():
        bp.reset(stream)
        bp.backproject(data, 0, w.n_views, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    rct.rct_profile_kernels(bp.ctx, True)
    l0 = bp.launches
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    kernel_ms, kernel_launches = rct.rct_profile_read(bp.ctx)
    rct.rct_profile_kernels(bp.ctx, False)
    launches = bp.launches - l0
    max_ms = dist.max(ms_total)
    total_updates = dist.sum(float(w.updates * args.steps))
    value = total_updates / (max_ms / 1e3) / 1e9

    # roofline of the dominant kernel (the backprojection pass).  The pass is bound by the L1TEX fetch
    # path, not by HBM: its fetch ceilings are measured live with the library's probes, with the lane
    # stride and z step of this workload (pixels per voxel at the isocentre).
    K = tun["views_per_pass"]
    n_launch = kernel_launches
    avg_kernel_s = kernel_ms / max(n_launch, 1) / 1e3
    passes_per_step = -(-w.n_views // K)
    upd_per_launch = w.updates / passes_per_step
    kernel_gups = upd_per_launch / avg_kernel_s / 1e9
    px_per_voxel = min(8.0, (w.geom.sdd / w.geom.sid) * float(w.spacing[0]) / w.geom.pitch)
    route = {rct.RCT_GATHER_LDG: "ldg", rct.RCT_GATHER_MIX: "mix", rct.RCT_GATHER_QUAD: "qld",
             rct.RCT_GATHER_PAIR: "pld"}.get(tun.get("gather"), "tex")
    probe = lambda mode, code=rct.RCT_PROJ_F32: round(
        probes.rct_probe_texture(mode, code, px_per_voxel, px_per_voxel, 4096) / 1e9, 1)
    fetch_probes = {"tex_tld4": probe(0), "ldg4": probe(3), "quad": probe(4), "pair": probe(5)}
    texel = 4 if args.dtype == "f32" else 2
    # The gather needs four texels (16 B FP32, 8 B 16-bit) per update from the L1/texture path.  Its
    # ceiling is the L1 load data path: 128 B per clock per SM x SMs x the SM clock measured during the run.
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    l1_derived = 128.0 * sms * sm_mhz * 1e6 / 1e9                     # GB/s
    # the same path measured in this run: coalesced 16-byte loads that hit L1, over every SM
    l1_peak = probes.rct_probe_l1_bandwidth(4096) / 1e9
    gather_gbs = kernel_gups * 4 * texel                              # GB/s of algorithmic texel bytes
    vol_bytes = 4 * w.L ** 3
    img_bytes = texel * w.geom.det_w * w.geom.det_h
    # per step: the first pass writes only, later passes read and write; each view's image is read once
    bytes_per_step = vol_bytes * (1 + 2 * (passes_per_step - 1)) + img_bytes * w.n_views
    bytes_per_launch = bytes_per_step / passes_per_step
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    achieved_gbs = bytes_per_launch / avg_kernel_s / 1e9
    rec = recorded_traffic(args.dtype, tun, w.L) if w.n_views == 496 else None
    traffic, traffic_src = (int(rec["bytes"]), rec["source"]) if rec else (None, None)
    # texture route: one tld4 gather per voxel update against the gather rate the probe measures for the
    # storage type of the step (the texture unit, not the load/store data path, fetches these cells)
    live = live_warp_fraction(w, tun)
    if route == "tex" and args.dtype != "f32":
        # BF16 is staged as 16-bit unsigned texels (there is no BF16 texture format); the probe's FP16
        # texels have the same size, which is what sets the gather rate
        tld4_peak = probe(0, codes["f16"])
        fetches = kernel_gups * live                                  # gathers issued per second (G/s)
        tex_view = {"achieved": round(fetches, 1), "peak": tld4_peak, "unit": "Gfetch/s",
                    "frac": round(fetches / tld4_peak, 4),
                    "what": "tld4 gathers issued: voxel updates of warps the clip test keeps",
                    "peak_source": "measured in this run: rct_probe_texture tld4 of 16-bit (FP16) texels"}
    else:
        tex_view = None
    # issue view: 4 warp instructions per clock per SM against the method's ~20 issue slots per voxel update
    # (3 incremental adds, reciprocal, 2 multiplies, floor and fraction, 3 lerps, r^2, accumulate, address math)
    issue_peak_gups = 4 * 32 * sms * sm_mhz * 1e6 / 20.0 / 1e9
    roofline = {"bound": "l1tex", "achieved": round(gather_gbs, 1), "peak": round(l1_peak, 1), "unit": "GB/s",
                "frac": round(gather_gbs / l1_peak, 4), "traffic": traffic,
                "traffic_source": (f"profiles/{traffic_src}: dram__bytes_read.sum + dram__bytes_write.sum of one "
                                   "accumulating launch of this kernel source and tuning") if traffic_src else
                                  "no capture of this kernel source and tuning",
                "what": (f"algorithmic gather bytes (four {args.dtype.upper()} texels per voxel update) through the "
                         "L1 load data path"),
                "peak_source": "measured in this run: rct_probe_l1_bandwidth (coalesced 16-byte loads that hit L1)",
                "peak_derived": {"value": round(l1_derived, 1), "frac": round(gather_gbs / l1_derived, 4),
                                 "source": f"128 B/clk/SM x {sms} SMs x {sm_mhz:.0f} MHz (median SM clock sampled "
                                           "during the timed region)"},
                "kernel": f"bp_kernel, {route} route", "kernel_gups": round(kernel_gups, 1),
                "kernel_share_of_step": round(kernel_ms / ms_total, 4), "updates_per_launch": int(upd_per_launch),
                "fetch_probes_gfetch_s": fetch_probes, "probe_lane_stride_px": round(px_per_voxel, 2),
                "issue": {"achieved": round(kernel_gups, 1), "peak": round(issue_peak_gups, 1), "unit": "GUPS",
                          "frac": round(kernel_gups / issue_peak_gups, 4),
                          "peak_source": "derived: 4 warp-instr/clk/SM x 32 lanes x SMs x SM clock / 20 issue slots "
                                         "per voxel update"},
                "live_warp_fraction": round(live, 4),
                "issued_gather_gbs": round(gather_gbs * live, 1),
                "tex": tex_view,
                "hbm": {"achieved": round(achieved_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                        "frac": round(achieved_gbs / hbm_peak, 4), "algorithmic_bytes_per_launch": int(bytes_per_launch),
                        "peak_source": "measured (MEASURED_PEAKS.json)" if "hbm_gbs" in peaks else "fallback"}}
    if rec and rec.get("lsu_wavefronts") and rec.get("updates"):
        # The unit that binds the load routes, counted: L1 data-pipe wavefronts (one per clock per SM at most).
        # ncu counts them for one launch of this kernel source and tuning; they scale with the launch's voxel
        # updates (the clip test keeps the same share of every view), so the average launch of the step
        # issues the recorded count x its updates / the recorded launch's updates, in the measured launch time.
        wf = rec["lsu_wavefronts"] * upd_per_launch / rec["updates"]
        wf_rate = wf / avg_kernel_s / 1e9
        wf_peak = sms * sm_mhz * 1e6 / 1e9
        roofline["l1_data_pipe"] = {
            "achieved": round(wf_rate, 1), "peak": round(wf_peak, 1), "unit": "Gwavefront/s",
            "frac": round(wf_rate / wf_peak, 4), "wavefronts_per_launch": int(wf),
            "wavefronts_per_update": round(wf / upd_per_launch, 3),
            "what": "L1 data-pipe wavefronts of the gather's loads (the count of an ncu capture, scaled to the "
                    "average launch) over the launch time measured in this run",
            "peak_source": f"derived: 1 wavefront/clk/SM x {sms} SMs x {sm_mhz:.0f} MHz (median SM clock sampled "
                           "during the timed region)",
            "count_source": f"profiles/{rec['source']}: l1tex__data_pipe_lsu_wavefronts.sum of a launch of "
                            f"{rec['updates']} voxel updates"}
    if route == "ldg" and args.dtype == "f32":
        # Plain loads of four 4-byte taps: where lanes land far apart (L=128: 10 px) the L1 data pipe's
        # wavefronts, not its bytes, bind.  The ceiling of this access pattern is measured by replaying the
        # kernel's own warp footprints (projected from the geometry) in an L1-resident image; the cells the
        # kernel fetches are the updates of warps the clip test keeps.
        pc = pattern_ceiling(w, tun)
        if pc:
            cells = kernel_gups * live                                # G cells/s
            roofline["gather_pattern"] = {
                "achieved": round(cells, 1), "peak": round(pc / 1e9, 1), "unit": "Gcell/s",
                "frac": round(cells / (pc / 1e9), 4),
                "what": "cells gathered (four 4-byte loads each) by warps the clip test keeps",
                "peak_source": "measured in this run: rct_probe_gather_pattern with the kernel's warp footprint "
                               "at 8 views of the scan (mean)"}
    if tex_view is not None:
        # the texture route's gathers go through the texture pipe, not the load data path: its issued-gather
        # rate against the measured tld4 rate is the headline figure; the byte view moves to a sub-object
        lsu = {k: roofline.pop(k) for k in ("achieved", "peak", "unit", "frac", "what", "peak_source")}
        roofline = dict({"bound": "l1tex", **{k: tex_view[k] for k in ("achieved", "peak", "unit", "frac", "what",
                                                                         "peak_source")}},
                        **{k: v for k, v in roofline.items() if k != "bound"}, lsu_bytes=lsu)

    result = {
        "metric": METRIC_BY_DTYPE[args.dtype], "value": round(value, 2), "unit": UNIT, "n_gpus": dist.world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": dict(workload_config(args.workload, w, args.dtype), tuning=tun, parallelism=f"replicas x{dist.world}",
                       l2="inputs larger than L2 (2.4 GB projections, volume >= 512 MB); no flush"),
        "roofline": roofline,
        "clocks": clk,
        "gpu_launches": int(launches),
    }
    if dist.world > 1:
        result["note"] = "N > 1: replicas of the timed step and e2e only; the single-GPU legs run at N = 1"

    # --- end to end through the public API with host buffers
    if not args.no_e2e:
        from paper_1401_7494_gb300 import hostmem
        pinned, vol_host = (hostmem.finish(b) for b in host_bufs)
        host_bufs = None
        for _ in range(max(1, args.warmup)):
            bp.reset(stream)
            bp.backproject_host_read(pinned, vol_host, 0, w.n_views, stream)
        torch.cuda.synchronize()
        vol_dev = torch.empty((w.L,) * 3, dtype=torch.float32, device=dev)

        def plain_copy_gbs():
            # plain copy rates on this host link, to read the end-to-end number against
            c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            c0.record(stream)
            data.copy_(pinned, non_blocking=True)
            c1.record(stream)
            vol_host.copy_(vol_dev, non_blocking=True)
            c2.record(stream)
            torch.cuda.synchronize()
            return {"h2d": round(pinned.numel() * pinned.element_size() / (c0.elapsed_time(c1) / 1e3) / 1e9, 1),
                    "d2h": round(vol_host.numel() * 4 / (c1.elapsed_time(c2) / 1e3) / 1e9, 1)}

        copy_before = plain_copy_gbs()
        # Some hosts slow this process's host-to-device reads for tens of seconds at a time (plain copies at
        # 2-55 GB/s instead of the link's 210, with no page migration or compaction on the host; the cause is
        # outside this process).  The timed region waits, up to LINK_WAIT_S, for a plain copy at half the
        # link's rate; the samples and the wait are reported beside the result.
        link_wait = wait_for_host_link(lambda: plain_copy_gbs()["h2d"], copy_before["h2d"])
        if link_wait["seconds"]:
            copy_before = plain_copy_gbs()
        e_steps = max(2, args.steps)
        dist.barrier()
        vm0 = vm_events()
        t0 = time.perf_counter()
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(e_steps + 1)]
        marks[0].record(stream)
        enqueue = []
        for i in range(e_steps):
            t_call = time.perf_counter()
            bp.reset(stream)
            bp.backproject_host_read(pinned, vol_host, 0, w.n_views, stream)
            enqueue.append((time.perf_counter() - t_call) * 1e3)
            marks[i + 1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        vm1 = vm_events()
        e_ms = max(marks[0].elapsed_time(marks[-1]), wall * 1e3)
        e_ms = dist.max(e_ms)
        in_order = [marks[i].elapsed_time(marks[i + 1]) for i in range(e_steps)]
        per_step = sorted(in_order)
        copy_after = plain_copy_gbs()
        # The same step captured once into a CUDA graph (rct_graph_*) and replayed: every replay still
        # copies the step's projections in and the volume out, but the host enqueues one launch per step.
        gs = torch.cuda.Stream(device=dev)
        bp.reset(gs)
        rct.rct_graph_begin(gs)
        try:
            bp.backproject_host_read(pinned, vol_host, 0, w.n_views, gs)
        finally:
            graph = rct.rct_graph_end(gs)
        try:
            for _ in range(max(1, args.warmup)):
                rct.rct_graph_launch(graph, gs)
            gs.synchronize()
            gmarks = [torch.cuda.Event(enable_timing=True) for _ in range(e_steps + 1)]
            t0 = time.perf_counter()
            gmarks[0].record(gs)
            for i in range(e_steps):
                rct.rct_graph_launch(graph, gs)
                gmarks[i + 1].record(gs)
            gs.synchronize()
            g_wall = time.perf_counter() - t0
        finally:
            rct.rct_graph_destroy(graph)
        g_ms = dist.max(max(gmarks[0].elapsed_time(gmarks[-1]), g_wall * 1e3))
        g_steps = [gmarks[i].elapsed_time(gmarks[i + 1]) for i in range(e_steps)]
        del vol_dev
        result["e2e"] = {"value": round(dist.sum(float(w.updates * e_steps)) / (e_ms / 1e3) / 1e9, 2), "unit": UNIT,
                         "h2d_bytes_per_step": int(pinned.numel() * pinned.element_size()),
                         "d2h_bytes_per_step": int(vol_host.numel() * 4),
                         "steps": e_steps,
                         "api": "rct_backproject_host_read (page-locked huge-page host buffers from hostmem.pinned_empty; "
                                "the volume read-back overlaps the last pass)",
                         "ms_per_step": round(e_ms / e_steps, 3)}
        e2e_detail = {"host_buffers_huge_page_fraction": {"projections": round(hostmem.huge_fraction(pinned), 3),
                                                          "volume": round(hostmem.huge_fraction(vol_host), 3),
                                                          "at_allocation": huge_at_allocation},
                      "step_ms": {"min": round(per_step[0], 3), "median": round(statistics.median(per_step), 3),
                                  "max": round(per_step[-1], 3), "in_order": [round(t, 2) for t in in_order]},
                      "host_enqueue_ms": [round(t, 2) for t in enqueue],
                      "plain_copy_gbs": {"before": copy_before, "after": copy_after},
                      "host_link_wait": link_wait,
                      # the host's page migration and compaction during the timed region (system-wide counters)
                      "host_vm_events": {k: vm1[k] - vm0[k] for k in vm1 if k in vm0} if vm0 and vm1 else None,
                      "graph_replay": {
                             "value": round(dist.sum(float(w.updates * e_steps)) / (g_ms / 1e3) / 1e9, 2),
                             "unit": UNIT, "ms_per_step": round(g_ms / e_steps, 3),
                             "api": "the same call captured once with rct_graph_begin/end, replayed with rct_graph_launch",
                             "step_ms": {"min": round(min(g_steps), 3), "median": round(statistics.median(g_steps), 3),
                                         "max": round(max(g_steps), 3), "in_order": [round(t, 2) for t in g_steps]}}}
        del pinned, vol_host

    bp.close()
    if dist.rank == 0:
        result["staging"] = {"convert": convert_leg(proj, stream, peaks)}
    host = proj.cpu().numpy() if dist.rank == 0 and not (args.no_variants and args.no_cpu_baseline) else None
    if dist.rank == 0 and not args.no_variants:
        L = w.L
        rng = np.random.default_rng(7)
        check_idx = np.unique(np.concatenate([rng.integers(0, L ** 3, size=8192),
                                              np.arange(L * L, dtype=np.int64) + (L // 2) * L * L]))
        import oracle
        variants = {}
        for dt, it, fr, tr in [("f32", "soft", "global", False), ("f32", "soft", "block", False),
                               ("f32", "soft", "global", True), ("f16", "soft", "global", False),
                               ("bf16", "soft", "global", False), ("f16", "tex", "global", False),
                               ("bf16", "tex", "global", False), ("f32", "tex", "global", False)]:
            # the error is stated against the FP64 oracle on the FP32 projections (with the same index rule)
            name = f"{dt}_{it}" + ("_block_frame" if fr == "block" else "") + ("_rabbitct_trunc" if tr else "")
            variants[name] = measure_variant(w, proj, dt, it, max(2, args.steps // 2), 1, stream,
                                             check_idx=check_idx, host=host, frame=fr, trunc=tr)
        result["variants"] = variants
        result["variants_note"] = ("GUPS per precision variant on the same workload; error vs the FP64 oracle on "
                                   f"FP32 projections over {check_idx.size} sampled voxels (a full z-plane + random)")

    del proj, data
    torch.cuda.empty_cache()
    if dist.rank == 0 and not args.no_prefilter:
        result["prefilter"] = prefilter_leg(args.workload, dev, stream, peaks, result["ms_per_step"])
        torch.cuda.empty_cache()
    if dist.rank == 0 and not args.no_k_sweep:
        result["k_sweep"] = k_sweep(dev, stream, peaks)
        torch.cuda.empty_cache()
    if dist.rank == 0 and not args.no_serve:
        from paper_1401_7494_gb300 import serve_bench
        protocols, host_data = serve_bench.build_protocols(dev, raw=True)
        # the requests' projections stream from page-locked host memory: the same bounded wait for a ready
        # host link as the end-to-end leg, before each mode
        probe_src = next(iter(host_data.values()))
        probe_dst = torch.empty(probe_src.shape, dtype=probe_src.dtype, device=dev)

        def probe_h2d() -> float:
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            probe_dst.copy_(probe_src, non_blocking=True)
            c1.record(stream)
            torch.cuda.synchronize()
            return probe_src.numel() * probe_src.element_size() / (c0.elapsed_time(c1) / 1e3) / 1e9

        served = {}
        for mode, raw in (("f32", False), ("f16", False), ("f16", True)):
            wait = wait_for_host_link(probe_h2d, probe_h2d())
            key = mode + ("_raw_ingest" if raw else "")
            served[key] = serve_bench.run_mode(
                mode, protocols, host_data, n_requests=args.serve_requests, raw=raw, log=lambda *_: None)
            served[key]["host_link_wait"] = wait
        del probe_dst
        result["served"] = {m: {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
                            for m, r in served.items()}
        del host_data

    if dist.rank == 0 and not args.no_cpu_baseline:
        gups, cores, sample = oracle_rate(w, host, args.cpu_seconds)
        one, one_sample = oracle_rate_one_core(w, host)
        result["cpu_baseline"] = {"value": round(gups, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                                  "sample": sample,
                                  "single_thread": {"value": round(one, 4), "unit": UNIT, "sample": one_sample}}
    if not args.no_e2e:
        result["e2e_detail"] = e2e_detail          # last key: it stays in the tail of a truncated log
    return result


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, dist: Dist) -> dict | None:
    if dist.rank != 0:
        return None
    import synth
    import oracle
    w = synth.workloads.named(args.workload)
    host = w.projections(device="cuda" if _cuda_ok() else "cpu").cpu().numpy()
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    rates = []
    step_ms = []
    cores = oracle.max_threads()
    sample = ""
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        gups, cores, sample = oracle_rate(w, host, per_step)
        if i >= args.warmup:
            rates.append(gups)
            step_ms.append((time.perf_counter() - t) * 1e3)
    value = statistics.median(rates)
    # A step is one bounded sample of the reconstruction (a slab of z-planes x all views, sized for
    # about per_step seconds); ms_per_step is the wall time those steps took, and the time a whole
    # reconstruction would take at the measured rate is given beside it.
    return {"metric": METRIC_BY_DTYPE[args.dtype], "value": round(value, 4), "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(statistics.median(step_ms), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": dict(workload_config(args.workload, w, args.dtype), per_step_sample=sample,
                           ms_per_whole_reconstruction=round(w.updates / (value * 1e9) * 1e3, 1)),
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _cuda_ok() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def main():
    args = parse_args()
    dist = Dist(args.gpus)
    try:
        if args.impl == "reference":
            res = run_reference(args, dist)
        else:
            res = run_ours(args, dist)
    finally:
        dist.close()
    if dist.rank == 0 and res is not None:
        line = json.dumps(res)
        print(line, flush=True)
        if args.out:
            Path(args.out).write_text(line + "\n")


if __name__ == "__main__":
    main()
