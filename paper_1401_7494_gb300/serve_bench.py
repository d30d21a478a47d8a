"""Serving benchmark: a Poisson stream of mixed reconstruction requests through the scheduler.

Requests: L in {128, 256, 512, 1024} with weights 0.4/0.3/0.2/0.1, scan
protocols of 124, 248 or 496 views of 1248 x 960 pixels, projections arriving
in chunks of 16 views at the detector rate ``views_per_s``; the arrival rate
is chosen for a target device load from the measured (autotuned) GUPS of
each L.  Reports served GUPS and p50/p99 time-to-volume.

Usage: python -m paper_1401_7494_gb300.serve_bench [--requests 200] [--mode f32 f16]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import hostmem, serving, tuning

PROTOCOL_VIEWS = {"short124": 124, "short248": 248, "short496": 496}
L_CHOICES = (128, 256, 512, 1024)
L_WEIGHTS = (0.4, 0.3, 0.2, 0.1)


def build_protocols(device, det_w=1248, det_h=960, seed=1405, raw=False):
    """Scan protocols (geometry) and pinned host projections of a seeded phantom for each: filtered
    (key: protocol name) and, with ``raw``, the raw line integrals too (key: name + "/raw")."""
    import torch
    import synth
    protocols, host = {}, {}
    for i, (name, n) in enumerate(sorted(PROTOCOL_VIEWS.items())):
        w = synth.make_workload(128, n_views=n, det_w=det_w, det_h=det_h, seed=seed + i)
        protocols[name] = serving.Protocol_(name, det_w, det_h, w.geom.matrices, w.geom.sdd, w.geom.pitch,
                                            w.geom.principal)
        kinds = [(name, dict())] + ([(name + "/raw", dict(weighted=False, filtered=False))] if raw else [])
        for key, kw in kinds:
            proj = synth.make_projections(w.geom, w.phantom, device=device, **kw)
            pinned = hostmem.pinned_empty(proj.shape, torch.float32)   # huge-page backed: no copy stalls
            pinned.copy_(proj)
            host[key] = pinned
            del proj
    torch.cuda.synchronize()
    return protocols, host


def expected_service_s(mode: str) -> float:
    """Mean device time per request from the autotuned GUPS of each L (no concurrency)."""
    mean_views = np.mean(list(PROTOCOL_VIEWS.values()))
    s = 0.0
    for L, wgt in zip(L_CHOICES, L_WEIGHTS):
        gups = _gups(L, mode)
        s += wgt * L ** 3 * mean_views / (gups * 1e9)
    return s


def _gups(L: int, mode: str) -> float:
    cache = tuning.load_cache()
    for gpu, entries in cache.items():
        for key in (f"L{L}/{mode}/soft",):
            if key in entries:
                return float(entries[key]["gups"])
    # interpolate from neighbours when an L was not tuned (e.g. 256)
    known = {}
    for gpu, entries in cache.items():
        for key, rec in entries.items():
            parts = key.split("/")
            if len(parts) != 3:               # frame-specific entries are not serving modes
                continue
            l, m, i = parts
            if m == mode and i == "soft":
                known[int(l[1:])] = float(rec["gups"])
    if known:
        ls = sorted(known)
        return float(np.interp(L, ls, [known[x] for x in ls]))
    return 500.0


def run_mode(mode: str, protocols, host, *, n_requests=200, load=0.7, views_per_s=2000.0, seed=2024,
             budget_gb=200.0, max_active=32, use_graphs=True, raw=False, log=print) -> dict:
    import torch
    svc = expected_service_s(mode)
    rate = load / svc
    reqs = serving.poisson_requests(n_requests, rate, PROTOCOL_VIEWS, seed=seed, L_choices=L_CHOICES,
                                    L_weights=L_WEIGHTS, mode=mode, views_per_s=views_per_s, raw=raw)
    ex = serving.GpuExecutor(protocols, host, use_graphs=use_graphs, timeline=True)
    sch = serving.Scheduler(ex, int(budget_gb * (1 << 30)), max_active=max_active)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = sch.run(reqs)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    out = serving.summarize(res, reqs, wall)
    live = peak = 0
    for _, ev, _ in sch.log:
        live += {"admit": 1, "done": -1, "timeout": -1}.get(ev, 0)
        peak = max(peak, live)
    out.update({"mode": mode, "raw_ingest": raw, "arrival_rate_hz": rate, "target_load": load, "expected_service_s": svc,
                "views_per_s": views_per_s, "graph_captures": ex.captures, "graph_launches": ex.graph_launches,
                "peak_concurrent_requests": peak, "offered_updates": sum(r.updates for r in reqs),
                "span_s": reqs[-1].arrival})
    # device evidence of overlap: CUDA-event intervals of every chunk's work on its request's stream
    ov = serving.overlap_stats(ex.device_timeline())
    out["device_overlap"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in ov.items()}
    ex.close()
    log(json.dumps(out))
    return out


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--mode", nargs="+", default=["f32", "f16"])
    ap.add_argument("--load", type=float, default=0.7)
    ap.add_argument("--views-per-s", type=float, default=2000.0)
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--raw", action="store_true", help="requests send raw line integrals (filtered on the device)")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    protocols, host = build_protocols(dev, raw=args.raw)
    results = {m: run_mode(m, protocols, host, n_requests=args.requests, load=args.load,
                           views_per_s=args.views_per_s, use_graphs=not args.no_graphs, raw=args.raw)
               for m in args.mode}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(results, f, indent=1)


if __name__ == "__main__":
    sys.exit(main())
