"""Autotuner for the backprojection launch: views per pass K, z-run, x-vector, block shape, gather kind.

Coordinate descent over the candidate lists, from several starts (the
built-in default and the current cache entries): each round varies one
parameter at a time, keeping the fastest value, until a round changes
nothing; the best end point wins.  Each candidate is timed with CUDA
events on a fixed run of views of the real workload (warm-up excluded), so
the winner is picked on GUPS for that (L, dtype, interpolation).  Results go
to the JSON cache read by ``tuning.lookup``.

Usage: python -m paper_1401_7494_gb300.autotune --L 512 [--dtype f32] [--interp soft]
"""
from __future__ import annotations

import argparse
import itertools
import json
import sys

from . import rct, tuning

CANDIDATES = {
    # (gather route, z positions per run through the texture gather when mixed)
    "gather": [(rct.RCT_GATHER_TLD4, 0), (rct.RCT_GATHER_LDG, 0), (rct.RCT_GATHER_QUAD, 0),
               (rct.RCT_GATHER_PAIR, 0), (rct.RCT_GATHER_DQUAD, 0), (rct.RCT_GATHER_MIX, 1), (rct.RCT_GATHER_MIX, 2),
               (rct.RCT_GATHER_MIX, 4), (rct.RCT_GATHER_MIX, 6)],
    "views_per_pass": [4, 8, 16, 24, 32],
    "zrun": [1, 2, 4, 8, 16],
    "xvec": [1, 2, 4],
    "block": [(32, 4), (32, 8), (32, 16), (64, 2), (64, 4), (16, 8), (16, 16), (8, 16), (128, 2)],
    "view_split": [1, 2, 4, 8],
}


def _valid(L: int, t: dict, dtype: str = "f32") -> bool:
    bx, by = t["block_x"], t["block_y"]
    if t.get("gather") == rct.RCT_GATHER_DQUAD and dtype != "f32":      # difference quads hold FP32 values
        return False
    if t.get("gather") == rct.RCT_GATHER_MIX and not (1 <= t.get("tex_zrun", 0) < t["zrun"]):
        return False
    if t["zrun"] == 16 and t["xvec"] > 2:
        return False
    if t.get("view_split", 1) > 1 and t.get("view_split", 1) > t["views_per_pass"]:
        return False
    return L % t["xvec"] == 0 and bx * by <= 512 and (bx * by) % 32 == 0


def search_params(interp: str, frame: str) -> list:
    """The tuning fields the descent varies.  Texture filtering has one gather; the view split runs only with
    software interpolation in the global frame (the library rejects it elsewhere)."""
    params = ["gather", "views_per_pass", "zrun", "xvec", "block", "view_split"]
    if interp == "tex":
        params.remove("gather")
    if interp == "tex" or frame == "block":
        params.remove("view_split")
    return params


def time_candidate(bp, data, n_views: int, stream, reps: int = 3) -> float:
    """Seconds per backprojection of n_views views (best of reps after one warm-up)."""
    import torch
    bp.reset(stream)
    bp.backproject(data[:n_views], 0, n_views, stream)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bp.reset(stream)
        bp.backproject(data[:n_views], 0, n_views, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return best


def confirm_best(trials: list, rate_fn, top: int = 3) -> tuple[dict, float, list]:
    """Re-rate the ``top`` fastest distinct tunings of a descent with ``rate_fn(tuning) -> GUPS`` (a longer
    run, e.g. the whole scan) and return (winner, its confirmed GUPS, [(tuning, descent GUPS, confirmed
    GUPS), ...]).  A short run can favour a shape whose K divides its view count; the long run decides."""
    ranked, keys = [], set()
    for tr in sorted(trials, key=lambda tr: -tr["gups"]):
        key = tuple(sorted(tr["tuning"].items()))
        if key not in keys:
            keys.add(key)
            ranked.append(tr)
        if len(ranked) == top:
            break
    rows = [(dict(tr["tuning"]), tr["gups"], rate_fn(dict(tr["tuning"]))) for tr in ranked]
    best = max(rows, key=lambda r: r[2])
    return best[0], best[2], rows


def autotune(w, data, dtype: str = "f32", interp: str = "soft", n_views: int | None = None,
             rounds: int = 3, log=print, frame: str = "global",
             confirm_data=None, confirm_views: int = 0) -> tuple[dict, float, list]:
    """Return (best tuning, its GUPS, trial log) for workload ``w`` with projections ``data`` on the device.
    With ``confirm_data`` (projections of ``confirm_views`` views), the three fastest tunings of the descent
    are timed again on that longer run and the fastest there wins (its GUPS is the returned rate)."""
    import torch
    stream = torch.cuda.current_stream()
    codes = {"f32": rct.RCT_PROJ_F32, "f16": rct.RCT_PROJ_F16, "bf16": rct.RCT_PROJ_BF16}
    n_views = n_views or min(w.n_views, 96)
    updates = w.L ** 3 * n_views
    # Coordinate descent stops in a local optimum (a route that wins at the default z-run can lose at the
    # z-run it leads to), so it runs from several starts: the built-in default and the current cache entries
    # (this key's, and for block frames the global frame's); the best end point wins.
    starts = [dict(tuning.DEFAULT)]
    for cand in (tuning.lookup(w.L, dtype, interp, frame=frame), tuning.lookup(w.L, dtype, interp)):
        if cand not in starts:
            starts.append(dict(cand))
    for st in starts:
        st.setdefault("view_split", 1)
        if w.L % st["xvec"]:
            st["xvec"] = 1
    trials = []
    seen = {}
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
        bp.set_precision(codes[dtype], rct.RCT_INTERP_SOFT if interp == "soft" else rct.RCT_INTERP_TEX)
        bp.set_frame(rct.RCT_FRAME_BLOCK if frame == "block" else rct.RCT_FRAME_GLOBAL)

        def measure(t: dict) -> float:
            key = tuple(sorted(t.items()))
            if key in seen:
                return seen[key]
            bp.set_tuning(**t)
            s = time_candidate(bp, data, n_views, stream)
            g = updates / s / 1e9
            seen[key] = g
            trials.append({"tuning": dict(t), "gups": g})
            log(f"  {t} -> {g:.1f} GUPS")
            return g

        params = search_params(interp, frame)
        best_all, cur_all = -1.0, None
        for cur in starts:
            best = measure(cur)
            for _ in range(rounds):
                changed = False
                for p in params:
                    for val in CANDIDATES[p]:
                        t = dict(cur)
                        if p == "block":
                            t["block_x"], t["block_y"] = val
                        elif p == "gather":
                            t["gather"], t["tex_zrun"] = val
                        else:
                            t[p] = val
                        if t == cur or not _valid(w.L, t, dtype):
                            continue
                        g = measure(t)
                        if g > best * 1.01:
                            best, cur, changed = g, t, True
                if not changed:
                    break
            if best > best_all:
                best_all, cur_all = best, cur
        if confirm_data is not None and confirm_views > 0:
            def long_rate(t: dict) -> float:
                bp.set_tuning(**t)
                return w.L ** 3 * confirm_views / time_candidate(bp, confirm_data, confirm_views, stream) / 1e9
            cur_all, best_all, rows = confirm_best(trials, long_rate)
            for t, g_short, g_long in rows:
                log(f"  confirm {t}: {g_short:.1f} GUPS on {n_views} views, {g_long:.1f} on {confirm_views}")
    return cur_all, best_all, trials


def main(argv=None):
    import torch
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", default=[512])
    ap.add_argument("--dtype", nargs="+", default=["f32"])
    ap.add_argument("--interp", nargs="+", default=["soft"])
    ap.add_argument("--views", type=int, default=96)
    ap.add_argument("--frame", choices=["global", "block"], default="global",
                    help="block: tune the block-frame kernels (FP32 software interpolation), starting from the "
                         "global-frame entry")
    ap.add_argument("--confirm-views", type=int, default=0,
                    help="re-time the three fastest tunings on this many views (e.g. the whole 496-view scan) "
                         "and keep the fastest there")
    ap.add_argument("--cache", default=str(tuning.CACHE))
    ap.add_argument("--log", default=None)
    args = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    results = []
    for L in args.L:
        w = synth.make_workload(L, seed=1402)
        n_load = max(args.views, min(args.confirm_views, w.n_views))
        proj = w.projections(device=dev, views=list(range(n_load)))
        for dtype, interp in itertools.product(args.dtype, args.interp):
            data = proj
            if dtype != "f32":
                tdt = {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
                code = {"f16": rct.RCT_PROJ_F16, "bf16": rct.RCT_PROJ_BF16}[dtype]
                data = torch.empty(proj.shape, dtype=tdt, device=dev)
                rct.rct_convert_projections(proj, data, proj.numel(), code, torch.cuda.current_stream())
            print(f"L={L} {dtype} {interp} {args.frame} frame:", flush=True)
            confirm = min(args.confirm_views, n_load)
            t, g, trials = autotune(w, data, dtype, interp, n_views=args.views, frame=args.frame,
                                    confirm_data=data if confirm > args.views else None, confirm_views=confirm)
            print(f"  best {t} -> {g:.1f} GUPS", flush=True)
            tuning.store(L, dtype, interp, t, g, path=args.cache, extra={"trials": len(trials)}, frame=args.frame)
            results.append({"L": L, "dtype": dtype, "interp": interp, "best": t, "gups": g, "trials": trials})
    if args.log:
        with open(args.log, "w") as f:
            json.dump(results, f, indent=1)


if __name__ == "__main__":
    sys.exit(main())
