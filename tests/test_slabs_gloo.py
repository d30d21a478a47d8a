"""z-slab sharding (the paper's split into independent voxel planes, Section "Implementation") on the CPU:
the slab assignment, and the read-back of two gloo ranks' slabs into one volume."""
import os
import socket
import sys
from pathlib import Path

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1401_7494_gb300 import slabs

ROOT = Path(__file__).resolve().parents[1]


@pytest.mark.parametrize("L,parts", [(512, 1), (512, 2), (512, 3), (512, 8), (1024, 8), (128, 8), (100, 3),
                                     (17, 2), (33, 4)])
def test_slab_ranges_cover_the_volume_in_aligned_balanced_slabs(L, parts):
    r = slabs.slab_ranges(L, parts)
    assert len(r) == parts
    z = 0
    for z0, zc in r:                      # contiguous, in rank order, covering [0, L) once
        assert z0 == z and zc >= 0
        z += zc
    assert z == L
    for z0, zc in r:                      # every boundary on a 16-plane block (the last ends at L)
        assert z0 % 16 == 0 or zc == 0
        assert (z0 + zc) % 16 == 0 or z0 + zc == L
    blocks = [-(-zc // 16) for _, zc in r]
    assert max(blocks) - min(blocks) <= 1  # balanced to one block
    assert all(b > 0 for b in blocks) == (-(-L // 16) >= parts)


def test_slab_plan_rejects_bad_ranks():
    with pytest.raises(ValueError):
        slabs.SlabPlan.for_rank(64, 2, 2)
    assert slabs.SlabPlan.for_rank(16, 1, 2).empty


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case():
    import synth
    return synth.make_workload(19, n_views=5, det_w=28, det_h=22, seed=91)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, str(ROOT))
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1401_7494_gb300 import slabs as sl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _case()
    proj = w.projections().numpy()
    plan = sl.SlabPlan.for_rank(w.L, rank, world, align=4)
    # The rank's share of the reconstruction: its planes only (the oracle stands in for its GPU here).
    local = oracle.backproject(w.L, w.geom.det_w, w.geom.det_h, w.geom.matrices, w.origin, w.spacing, proj,
                               z_range=(plan.z_first, plan.z_first + plan.z_count))
    local = torch.from_numpy(local)
    dst = torch.full((w.L,) * 3, float("nan"), dtype=torch.float64) if rank == 0 else None
    got = sl.gather_slabs(local, plan, dst=dst)
    if rank == 0:
        out["volume"] = got.numpy().copy()
    out[f"plan{rank}"] = (plan.z_first, plan.z_count)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_gather_their_slabs_into_the_whole_volume(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        ps = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(timeout=180)
        assert all(p.exitcode == 0 for p in ps), [p.exitcode for p in ps]
        res = dict(out)
    import oracle
    w = _case()
    whole = oracle.backproject(w.L, w.geom.det_w, w.geom.det_h, w.geom.matrices, w.origin, w.spacing,
                               w.projections().numpy())
    plans = [res[f"plan{r}"] for r in range(world)]
    assert plans == slabs.slab_ranges(w.L, world, align=4)
    assert all(zc > 0 for _, zc in plans)
    assert np.array_equal(res["volume"], whole)     # planes are independent: the split changes no sum
