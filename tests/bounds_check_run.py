"""Run the backprojection through the bounds-checking build of the library and report violations.

Started by test_gpu_bounds_check.py in a subprocess with RCT_BUILD_VARIANT=check (the binding then
builds and loads that variant).  Prints one JSON line: the number of configurations run, the total
violation count, and the worst parity error against the oracle over the configurations it checks.
"""
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import synth  # noqa: E402
from paper_1401_7494_gb300 import build, rct  # noqa: E402
from gpu_helpers import oracle_volume, rel_errors  # noqa: E402


def main():
    assert build.VARIANT == "check", build.VARIANT
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    cases = {
        "L37": synth.make_workload(37, n_views=20, det_w=96, det_h=74, seed=21),
        "L40": synth.make_workload(40, n_views=33, det_w=130, det_h=100, seed=22),
        "L1": synth.make_workload(1, n_views=5, det_w=40, det_h=30, seed=31),
    }
    far = synth.make_workload(12, n_views=5, det_w=40, det_h=30, seed=40)
    far.origin = far.origin + np.array([0.0, 0.0, 5000.0])          # the whole volume off the detector
    cases["far"] = far
    G = rct
    tunings = []
    for gather in (G.RCT_GATHER_TLD4, G.RCT_GATHER_LDG, G.RCT_GATHER_QUAD, G.RCT_GATHER_PAIR, G.RCT_GATHER_MIX,
                   G.RCT_GATHER_DQUAD):
        for zrun, xvec in ((1, 1), (2, 2), (4, 4), (8, 1), (16, 2)):
            tunings.append(dict(gather=gather, zrun=zrun, xvec=xvec, tex_zrun=1, views_per_pass=7,
                                block_x=16, block_y=8))
    runs, violations, worst = 0, 0, 0.0
    for name, w in cases.items():
        proj = w.projections(device=dev)
        host = proj.cpu().numpy()
        ref = oracle_volume(w, host)
        for t in tunings:
            t = dict(t)
            if w.L % t["xvec"]:
                t["xvec"] = 1
            for frame, rule in ((G.RCT_FRAME_GLOBAL, G.RCT_INDEX_FLOOR), (G.RCT_FRAME_BLOCK, G.RCT_INDEX_FLOOR),
                                (G.RCT_FRAME_GLOBAL, G.RCT_INDEX_TRUNC)):
                with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
                    bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_frame(frame).set_index_rule(rule)
                    bp.set_tuning(**t)
                    out = torch.empty((w.L,) * 3, dtype=torch.float32, device=dev)
                    if t["zrun"] == 4:            # host input with the overlapped read-back
                        bp.backproject_host_read(proj.cpu().pin_memory(), out, 0, w.n_views, stream)
                    else:
                        bp.backproject(proj, 0, w.n_views, stream)
                        bp.read_volume(out, stream)
                    violations += rct.rct_debug_bound_violations(bp.ctx)
                    runs += 1
                    if rule == G.RCT_INDEX_FLOOR and np.any(ref != 0):
                        worst = max(worst, rel_errors(out.cpu().numpy(), ref)[0])
        # 16-bit storage through every route
        for dt in (G.RCT_PROJ_F16, G.RCT_PROJ_BF16):
            tdt = torch.float16 if dt == G.RCT_PROJ_F16 else torch.bfloat16
            data = torch.empty(proj.shape, dtype=tdt, device=dev)
            rct.rct_convert_projections(proj, data, proj.numel(), dt, stream)
            for gather in (G.RCT_GATHER_TLD4, G.RCT_GATHER_LDG, G.RCT_GATHER_QUAD, G.RCT_GATHER_PAIR):
                with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
                    bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_precision(dt, G.RCT_INTERP_SOFT)
                    bp.set_tuning(gather=gather, zrun=8, xvec=1, views_per_pass=9)
                    bp.backproject(data, 0, w.n_views, stream)
                    violations += rct.rct_debug_bound_violations(bp.ctx)
                    runs += 1
    # Slab contexts: every plane index stays inside the slab's own buffer, through the device and host paths.
    w = cases["L40"]
    proj = w.projections(device=dev)
    for z0, zc in ((0, 16), (16, 16), (32, 8), (16, 24)):
        for gather, zrun in ((G.RCT_GATHER_PAIR, 16), (G.RCT_GATHER_DQUAD, 8), (G.RCT_GATHER_LDG, 4)):
            with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views, z_range=(z0, zc)) as bp:
                bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
                bp.set_tuning(gather=gather, zrun=zrun, xvec=1, views_per_pass=7)
                out = torch.empty((zc, w.L, w.L), dtype=torch.float32, device=dev)
                if zrun == 4:
                    bp.backproject_host_read(proj.cpu().pin_memory(), out, 0, w.n_views, stream)
                else:
                    bp.backproject(proj, 0, w.n_views, stream)
                    bp.read_volume(out, stream)
                violations += rct.rct_debug_bound_violations(bp.ctx)
                runs += 1
    # Control: with the bounds checks' staged-image limit lowered to a tenth of the image, in-bounds pair loads
    # past it are counted (and skipped); restored, the count stops growing.
    w = cases["L40"]
    proj = w.projections(device=dev)
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(gather=G.RCT_GATHER_PAIR, zrun=4)
        pair_elems = (w.geom.det_w + 2) * (w.geom.det_h + 1)
        rct.rct_debug_lower_bound_limit(bp.ctx, pair_elems // 10)
        bp.backproject(proj, 0, w.n_views, stream)
        control = rct.rct_debug_bound_violations(bp.ctx)
        rct.rct_debug_lower_bound_limit(bp.ctx, 0)
        bp.backproject(proj, 0, w.n_views, stream)
        control_after = rct.rct_debug_bound_violations(bp.ctx)
    print(json.dumps({"runs": runs, "violations": violations, "worst_rel_rms": worst, "control": control,
                      "control_after_restore": control_after}))


if __name__ == "__main__":
    main()
