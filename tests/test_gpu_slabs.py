"""Slab contexts (rct_create_slab): the paper's split of the volume into independent voxel planes
(Section "Implementation") as the unit of work of one GPU.  Two slab contexts on one GPU stand in for
two ranks: together they reproduce the whole-volume context bit for bit and the FP64 oracle within the
FP32 bar (needs a GPU)."""
import numpy as np
import pytest
import torch

import synth
from paper_1401_7494_gb300 import rct, slabs
from gpu_helpers import assert_parity, gpu_backproject, oracle_volume

pytestmark = pytest.mark.gpu

TUNES = [dict(gather=rct.RCT_GATHER_PAIR, views_per_pass=16, zrun=8, xvec=1, block_x=8, block_y=16),
         dict(gather=rct.RCT_GATHER_PAIR, views_per_pass=9, zrun=16, xvec=1, block_x=8, block_y=16),
         dict(gather=rct.RCT_GATHER_TLD4, views_per_pass=7, zrun=4, xvec=2, block_x=16, block_y=8),
         dict(gather=rct.RCT_GATHER_LDG, views_per_pass=32, zrun=2, xvec=1, block_x=32, block_y=4),
         dict(gather=rct.RCT_GATHER_LDG, views_per_pass=12, zrun=4, xvec=1, block_x=8, block_y=16, view_split=4)]


@pytest.fixture(scope="module")
def case(cuda_device):
    w = synth.make_workload(44, n_views=29, det_w=130, det_h=100, seed=71)   # 44 = 16 + 16 + 12: ragged slab
    proj = w.projections(device=cuda_device)
    return w, proj, oracle_volume(w, proj.cpu().numpy())


def _slab_volume(w, proj, z_first, z_count, tuning, host_read=False):
    stream = torch.cuda.current_stream()
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views, z_range=(z_first, z_count)) as bp:
        assert rct.rct_get_slab(bp.ctx) == (z_first, z_count)
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**tuning)
        out = torch.empty((z_count, w.L, w.L), dtype=torch.float32, pin_memory=host_read,
                          device=None if host_read else proj.device)
        if host_read:
            host = proj.cpu().pin_memory()
            bp.reset(stream)
            bp.backproject_host_read(host, out, 0, w.n_views, stream)
        else:
            bp.reset(stream)
            bp.backproject(proj[:11], 0, 11, stream)            # two calls: accumulate across calls
            bp.backproject(proj[11:], 11, w.n_views - 11, stream)
            bp.read_volume(out, stream)
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("ti", range(len(TUNES)))
@pytest.mark.parametrize("parts", [2, 3])
def test_aligned_slabs_reproduce_the_whole_volume_bitwise(case, ti, parts):
    w, proj, ref = case
    whole = gpu_backproject(w, proj, tuning=TUNES[ti], chunks=[(0, 11), (11, w.n_views)])
    got = np.concatenate([_slab_volume(w, proj, z0, zc, TUNES[ti])
                          for z0, zc in slabs.slab_ranges(w.L, parts)], axis=0)
    assert got.shape == whole.shape
    assert np.array_equal(got, whole), f"slabs differ from the whole volume at {np.argwhere(got != whole)[:3]}"
    assert_parity(got, ref, f"{parts} slabs, tuning {TUNES[ti]}")


def test_slab_boundaries_must_be_aligned(cuda_device):
    """A z-run never crosses a slab boundary: boundaries lie on multiples of 16 planes (the end may be L)."""
    for z0, zc in [(5, 13), (0, 20), (8, 8), (16, 20)]:
        with pytest.raises(rct.RctError) as e:
            rct.rct_create_slab(44, 64, 48, 4, z0, zc)
        assert e.value.status == rct.RCT_EINVAL and "multiples" in rct.rct_last_error()
    for z0, zc in [(0, 16), (16, 28), (32, 12), (0, 44)]:
        rct.rct_destroy(rct.rct_create_slab(44, 64, 48, 4, z0, zc))


@pytest.mark.parametrize("z_first,z_count", [(0, 16), (16, 28), (32, 12)])
def test_slab_host_read_equals_the_device_path(case, z_first, z_count):
    w, proj, ref = case
    dev = _slab_volume(w, proj, z_first, z_count, TUNES[0])
    host = _slab_volume(w, proj, z_first, z_count, TUNES[0], host_read=True)
    # the host path passes views in batches of K from the first; the device path above splits at view 11,
    # so the two sum the same terms in different batches: compare both with the oracle, and each other
    assert_parity(host, ref[z_first:z_first + z_count], f"host-read slab [{z_first}, {z_first + z_count})")
    assert_parity(dev, host, "device vs host slab")


def test_slab_range_errors(cuda_device):
    for z0, zc in [(-1, 4), (0, 0), (40, 5), (3, 42)]:
        with pytest.raises(rct.RctError) as e:
            rct.rct_create_slab(44, 64, 48, 4, z0, zc)
        assert e.value.status == rct.RCT_EINVAL


def test_slab_buffers_are_checked_against_the_slab(case):
    w, proj, _ = case
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views, z_range=(16, 16)) as bp:
        small = torch.empty((15, w.L, w.L), dtype=torch.float32, device=proj.device)
        with pytest.raises(ValueError):
            bp.read_volume(small)
        ok = torch.empty((16, w.L, w.L), dtype=torch.float32, device=proj.device)
        bp.read_volume(ok)
        torch.cuda.synchronize()
        assert float(ok.abs().max()) == 0.0          # a fresh context reads back zeros
