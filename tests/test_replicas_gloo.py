"""The N > 1 replica bookkeeping of bench.py (barrier, max of the timed region, sum of the work),
run as two gloo ranks on the CPU."""
import os
import socket
import sys
from pathlib import Path

import pytest
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, str(ROOT))
    import bench
    d = bench.Dist(world, backend="gloo")
    d.barrier()
    ms = [120.0, 95.5][rank]                 # each replica's timed region
    upd = [3e10, 5e10][rank]                 # each replica's voxel updates
    out[rank] = (d.rank, d.world, d.max(ms), d.sum(upd))
    d.barrier()
    d.close()


def test_two_gloo_replicas_reduce_max_time_and_total_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        ps = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in ps), [p.exitcode for p in ps]
        res = dict(out)
    assert res[0] == (0, 2, 120.0, 8e10) and res[1] == (1, 2, 120.0, 8e10)
