"""The allocation-free entry point (for callers that cannot allocate device memory) gives the
same volume as the context-based entry point, on two calls in a row.

Kept in a file of its own, collected last, so a stop-at-first-failure run has already run every
other test before this one.  It needs nothing from earlier tests and also passes alone.
"""
import numpy as np
import pytest
import torch

import synth
from paper_1401_7494_gb300 import rct
from gpu_helpers import assert_parity, gpu_backproject, oracle_inputs, oracle_volume

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_entry_point_twice(cuda_device):
    w = synth.make_workload(40, n_views=45, det_w=131, det_h=97, seed=61)   # odd sizes: unaligned view offsets
    proj = w.projections(device=cuda_device)
    # existing entry point: a context with FP16 storage and the same kernel shape
    ref = gpu_backproject(w, proj, dtype="f16",
                          tuning=dict(gather=rct.RCT_GATHER_LDG, views_per_pass=32, zrun=4, xvec=1,
                                      block_x=32, block_y=8))
    # and the FP64 oracle fed the same FP16-rounded projections
    truth = oracle_volume(w, oracle_inputs(proj.cpu().numpy(), "f16"))
    stream = torch.cuda.current_stream()
    vol = torch.full((w.L,) * 3, 123.0, dtype=torch.float32, device=cuda_device)   # overwritten, not added to
    for call in range(2):
        rct.rct_backproject_f16_noalloc(w.L, w.geom.det_w, w.geom.det_h, w.geom.matrices, w.origin, w.spacing,
                                        proj, w.n_views, vol, accumulate=False, stream=stream)
        torch.cuda.synchronize()
        got = vol.cpu().numpy()
        assert_parity(got, ref, f"no-alloc call {call + 1} vs the context entry point")
        assert_parity(got, truth, f"no-alloc call {call + 1} vs the oracle")


def test_noalloc_accumulates_over_split_views(cuda_device):
    """Two calls over views [0, 20) and [20, 45), the second with accumulate=1, give the whole scan."""
    w = synth.make_workload(40, n_views=45, det_w=131, det_h=97, seed=62)
    proj = w.projections(device=cuda_device)
    truth = oracle_volume(w, oracle_inputs(proj.cpu().numpy(), "f16"))
    stream = torch.cuda.current_stream()
    vol = torch.full((w.L,) * 3, -7.0, dtype=torch.float32, device=cuda_device)
    m = w.geom.matrices
    rct.rct_backproject_f16_noalloc(w.L, w.geom.det_w, w.geom.det_h, m[:20], w.origin, w.spacing,
                                    proj[:20], 20, vol, accumulate=False, stream=stream)
    rct.rct_backproject_f16_noalloc(w.L, w.geom.det_w, w.geom.det_h, m[20:], w.origin, w.spacing,
                                    proj[20:], 25, vol, accumulate=True, stream=stream)
    torch.cuda.synchronize()
    assert_parity(vol.cpu().numpy(), truth, "split no-alloc calls vs the oracle")


def test_noalloc_rejects_a_view_larger_than_its_scratch(cuda_device):
    w = synth.make_workload(8, n_views=1, det_w=16, det_h=16, seed=1)
    vol = torch.zeros((8, 8, 8), device=cuda_device)
    # raw addresses: the library's own size checks, before any work is enqueued
    with pytest.raises(rct.RctError) as e:
        rct.rct_backproject_f16_noalloc(8, 5000, 4000, w.geom.matrices, w.origin, w.spacing,
                                        vol.data_ptr(), 1, vol.data_ptr(), stream=torch.cuda.current_stream())
    assert e.value.status == rct.RCT_EINVAL and "scratch" in str(e.value)
    # a row longer than the device's texture-gather extent (the limit rct_create takes)
    with pytest.raises(rct.RctError) as e:
        rct.rct_backproject_f16_noalloc(8, 40000, 1, w.geom.matrices, w.origin, w.spacing,
                                        vol.data_ptr(), 1, vol.data_ptr(), stream=torch.cuda.current_stream())
    assert e.value.status == rct.RCT_EINVAL and "exceeds" in str(e.value)
    # and the binding refuses a tensor too small for the view
    with pytest.raises(ValueError):
        rct.rct_backproject_f16_noalloc(8, 5000, 4000, w.geom.matrices, w.origin, w.spacing,
                                        vol, 1, vol, stream=torch.cuda.current_stream())
