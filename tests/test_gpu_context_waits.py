"""Set-up calls that replace a context's device state wait for that context's queued work only: a
geometry or filter change on one context (one serving slot) does not wait for another context's
passes still running on the device (needs a GPU)."""
import time

import numpy as np
import pytest
import torch

import synth
from paper_1401_7494_gb300 import rct, tuning
from gpu_helpers import assert_parity, gpu_backproject, oracle_volume

pytestmark = pytest.mark.gpu


def _busy_context(device):
    """A context whose backprojection keeps the device busy for about 50 ms (L = 512 x 496 full-size
    views, random projections -- the pass time does not depend on the values; 124 images serve the
    four quarters of the scan)."""
    geom = synth.short_scan(496, 1248, 960, pitch=0.308, seed=5)
    origin, spacing = synth.volume_grid(512)
    proj = torch.randn((124, 960, 1248), device=device)
    bp = rct.Backprojector(512, 1248, 960, 496)
    bp.set_geometry(geom.matrices, origin, spacing).set_tuning(**tuning.lookup(512, "f32", "soft"))
    return bp, proj


def test_set_geometry_does_not_wait_for_another_contexts_passes(cuda_device):
    busy, busy_proj = _busy_context(cuda_device)
    s_busy = torch.cuda.Stream(device=cuda_device)
    w = synth.make_workload(24, n_views=8, det_w=96, det_h=74, seed=3)
    proj = w.projections(device=cuda_device)
    other = synth.make_workload(24, n_views=8, det_w=96, det_h=74, seed=4)
    try:
        with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
            bp.set_geometry(other.geom.matrices, other.origin, other.spacing)
            bp.reset()
            bp.backproject(proj, 0, w.n_views)            # this context has launched work (on the legacy stream)
            torch.cuda.synchronize()
            def busy_step():
                busy.reset(s_busy)
                for q in range(4):
                    busy.backproject(busy_proj, 124 * q, 124, s_busy)
            busy_step()                                   # warm the busy context's staging
            s_busy.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s_busy)
            busy_step()
            e1.record(s_busy)
            t = time.perf_counter()
            bp.set_geometry(w.geom.matrices, w.origin, w.spacing)                       # replaces a table
            bp.set_filter(w.geom.sdd, w.geom.pitch, w.geom.principal)                   # replaces tables
            host_ms = (time.perf_counter() - t) * 1e3
            still_running = not s_busy.query()
            s_busy.synchronize()
            busy_ms = e0.elapsed_time(e1)
            assert busy_ms > 30.0, f"the busy pass took only {busy_ms:.1f} ms"
            assert still_running, (f"set-up calls on one context waited for another context's pass "
                                   f"({host_ms:.1f} ms of set-up, {busy_ms:.1f} ms pass)")
            # and the context still computes the new geometry correctly
            bp.reset()
            bp.backproject(proj, 0, w.n_views)
            out = torch.empty((w.L,) * 3, device=cuda_device)
            bp.read_volume(out)
            torch.cuda.synchronize()
            assert_parity(out.cpu().numpy(), oracle_volume(w, proj.cpu().numpy()), "after the geometry change")
    finally:
        busy.close()


def test_set_geometry_waits_for_its_own_queued_passes(cuda_device):
    """The block-frame table a queued pass reads is not overwritten under it: a geometry change right
    after enqueueing a pass leaves that pass's result equal to the old geometry's."""
    w = synth.make_workload(48, n_views=24, det_w=130, det_h=100, seed=8)
    other = synth.make_workload(48, n_views=24, det_w=130, det_h=100, seed=9)
    proj = w.projections(device=cuda_device)
    s = torch.cuda.Stream(device=cuda_device)
    ref = gpu_backproject(w, proj, frame=rct.RCT_FRAME_BLOCK)
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_frame(rct.RCT_FRAME_BLOCK).set_geometry(w.geom.matrices, w.origin, w.spacing)
        out = torch.empty((w.L,) * 3, device=cuda_device)
        bp.reset(s)
        bp.backproject(proj, 0, w.n_views, s)
        bp.read_volume(out, s)
        bp.set_geometry(other.geom.matrices, other.origin, other.spacing)
        s.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
