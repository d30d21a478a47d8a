"""Serving on the GPU: results are the same alone and in a concurrent mix, and match the oracle."""
import numpy as np
import pytest
import torch

import synth
from paper_1401_7494_gb300 import serving
from gpu_helpers import assert_parity, oracle_volume, oracle_inputs

pytestmark = pytest.mark.gpu

W, H = 160, 123


@pytest.fixture(scope="module")
def setup(cuda_device):
    protos, host, works = {}, {}, {}
    for name, n, seed in [("pA", 24, 51), ("pB", 40, 52)]:
        w = synth.make_workload(32, n_views=n, det_w=W, det_h=H, seed=seed)
        protos[name] = serving.Protocol_(name, W, H, w.geom.matrices, w.geom.sdd, w.geom.pitch, w.geom.principal)
        p = w.projections(device=cuda_device)
        host[name] = p.cpu().pin_memory()
        raw = synth.make_projections(w.geom, w.phantom, device=cuda_device, weighted=False, filtered=False)
        host[name + "/raw"] = raw.cpu().pin_memory()
        works[name] = w
    return protos, host, works


def _req(rid, L, proto, n, arrival, mode="f32", interval=0.0, raw=False):
    sp = 256.0 / L
    return serving.Request(rid, L, proto, n, arrival, mode, chunk_views=16, chunk_interval=interval,
                           origin=(-(L - 1) / 2 * sp,) * 3, spacing=(sp,) * 3, raw=raw)


def _serve(protos, host, reqs, graphs=True):
    ex = serving.GpuExecutor(protos, host, use_graphs=graphs)
    sch = serving.Scheduler(ex, 8 << 30, max_active=8, keep_volumes=True)
    res = sch.run(reqs)
    stats = (ex.captures, ex.graph_launches)
    ex.close()
    return res, stats


@pytest.mark.parametrize("mode", ["f32", "f16"])
def test_alone_equals_in_the_mix_and_matches_oracle(setup, mode):
    protos, host, works = setup
    target = _req(0, 37, "pB", 40, 0.0, mode)
    alone, _ = _serve(protos, host, [target])
    assert alone[0].status == "ok"
    mix = [_req(0, 37, "pB", 40, 0.002, mode, interval=0.001)]
    mix += [_req(i, L, p, n, 0.0005 * i, mode, interval=0.0007)
            for i, (L, p, n) in enumerate([(24, "pA", 24), (48, "pB", 40), (37, "pB", 40), (24, "pA", 24),
                                           (64, "pA", 24), (37, "pA", 24)], start=1)]
    res, (captures, launches) = _serve(protos, host, mix)
    assert all(r.status == "ok" for r in res)
    assert torch.equal(res[0].volume, alone[0].volume), "result changed when served in a mix"
    assert launches == sum(q.n_chunks for q in mix) and captures <= launches
    # and it is a correct reconstruction
    w = works["pB"]
    w37 = synth.Workload("t", 37, w.geom, np.array(target.origin), np.array(target.spacing), w.phantom, w.seed)
    ref = oracle_volume(w37, oracle_inputs(host["pB"].numpy(), "f16" if mode == "f16" else "f32"))
    assert_parity(res[0].volume.numpy(), ref, f"served {mode}")


def test_graph_and_direct_paths_agree(setup):
    protos, host, _ = setup
    reqs = [_req(0, 40, "pA", 24, 0.0), _req(1, 40, "pA", 24, 0.0)]
    g, _ = _serve(protos, host, reqs, graphs=True)
    d, _ = _serve(protos, host, reqs, graphs=False)
    for a, b in zip(g, d):
        assert torch.equal(a.volume, b.volume)


def test_slots_and_graphs_are_reused_across_requests(setup):
    protos, host, _ = setup
    reqs = [_req(0, 40, "pB", 40, 0.0), _req(1, 40, "pB", 40, 0.5)]      # same shape, one after the other
    res, (captures, launches) = _serve(protos, host, reqs)
    assert [r.status for r in res] == ["ok", "ok"]
    assert captures == reqs[0].n_chunks and launches == 2 * reqs[0].n_chunks
    assert torch.equal(res[0].volume, res[1].volume)


@pytest.mark.parametrize("mode", ["f32", "f16"])
def test_raw_ingest_filters_on_the_device(setup, mode, cuda_device):
    """A request that sends raw line integrals gets the same volume, bit for bit, as one that sends
    the device filter's output (computed up front through rct_filter_projections), alone and in a mix."""
    from paper_1401_7494_gb300 import rct
    protos, host, works = setup
    p, w = protos["pB"], works["pB"]
    raw_dev = host["pB/raw"].to(cuda_device)
    filt = torch.empty_like(raw_dev)
    with rct.Backprojector(8, W, H, w.n_views) as bp:
        bp.set_filter(p.sdd, p.pitch, p.principal)
        bp.filter(raw_dev, filt)
        torch.cuda.synchronize()
    host2 = dict(host, pF=filt.cpu().pin_memory())
    protos2 = dict(protos, pF=serving.Protocol_("pF", W, H, p.matrices, p.sdd, p.pitch, p.principal))
    pre, _ = _serve(protos2, host2, [_req(0, 37, "pF", 40, 0.0, mode)])
    mix = [_req(0, 37, "pB", 40, 0.001, mode, interval=0.001, raw=True),
           _req(1, 24, "pA", 24, 0.0, mode, interval=0.0007),
           _req(2, 48, "pB", 40, 0.0005, mode, interval=0.0007, raw=True)]
    res, _ = _serve(protos2, host2, mix)
    assert all(r.status == "ok" for r in res)
    assert torch.equal(res[0].volume, pre[0].volume)


def test_raw_ingest_needs_filter_geometry(setup):
    protos, host, _ = setup
    bare = dict(protos, pX=serving.Protocol_("pX", W, H, protos["pA"].matrices))
    host2 = dict(host, **{"pX/raw": host["pA/raw"]})
    res, _ = _serve(bare, host2, [_req(0, 24, "pX", 24, 0.0, raw=True)])
    assert res[0].status == "error"


def test_concurrent_requests_overlap_on_the_device(setup, cuda_device):
    """Continuous batching puts different requests' work on the device at the same time: once the requests'
    slots exist (a first batch of the same shapes), the CUDA-event intervals of the chunks' work on their
    requests' streams overlap for a good part of the busy time."""
    protos, host, _ = setup
    # volumes large enough that a chunk's device work outlasts the host's submission of the next one
    shapes = [(256, "pB", 40), (256, "pB", 40), (224, "pA", 24), (256, "pB", 40), (224, "pA", 24), (256, "pB", 40)]
    ex = serving.GpuExecutor(protos, host, use_graphs=True)
    sch = serving.Scheduler(ex, 8 << 30, max_active=8)
    warm = sch.run([_req(i, L, p, n, 0.0, "f32") for i, (L, p, n) in enumerate(shapes)])
    assert all(r.status == "ok" for r in warm)
    ex.start_timeline()
    reqs = [_req(10 + i, L, p, n, 0.0, "f32") for i, (L, p, n) in enumerate(shapes)]
    res = serving.Scheduler(ex, 8 << 30, max_active=8).run(reqs)
    tl = ex.device_timeline()
    ex.close()
    assert all(r.status == "ok" for r in res)
    assert len(tl) == sum(q.n_chunks for q in reqs) and all(b >= a for _, _, a, b in tl)
    st = serving.overlap_stats(tl)
    assert st["peak_requests_in_flight"] >= 3 and st["overlap_fraction"] > 0.5, st
