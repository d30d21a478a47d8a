"""Parity at the measured configurations: 496 views of 1248x960, L = 128 and 512 (every voxel) and
L = 512 / 1024 (sampled voxels and whole planes), in the launch configuration the benchmark uses."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1401_7494_gb300 import rct
from paper_1401_7494_gb300 import tuning as tuning_mod
from gpu_helpers import assert_parity, gpu_backproject, oracle_volume, DTYPES, stored, oracle_inputs

pytestmark = pytest.mark.gpu


def _sampled_reference(w, host, idx):
    return oracle.backproject_voxels(w.L, w.geom.det_w, w.geom.det_h, w.geom.matrices, w.origin, w.spacing,
                                     host, idx, n_threads=oracle.max_threads())


def _sample_indices(L, seed, n_random=1 << 15, planes=(0,)):
    rng = np.random.default_rng(seed)
    idx = [rng.integers(0, L ** 3, size=n_random)]
    for z in planes:
        idx.append(np.arange(L * L, dtype=np.int64) + z * L * L)
    # the last row of the last plane: ragged x/y tails of the grid
    idx.append(np.arange(L, dtype=np.int64) + (L - 1) * L * L + (L - 1) * L)
    return np.unique(np.concatenate(idx))


def test_full_parity_L512_496_views(cuda_device):
    """The benchmark's workload and launch configuration, every one of the 512^3 voxels against the FP64
    oracle (about 45 s of oracle work on 16 host cores)."""
    w = synth.workloads.named("fp32_L512")
    proj = w.projections(device=cuda_device)
    host = proj.cpu().numpy()
    got = gpu_backproject(w, proj, tuning=tuning_mod.lookup(w.L, "f32", "soft"))
    del proj
    ref = oracle_volume(w, host)
    assert_parity(got, ref, "L=512 x 496 full volume")


def test_full_parity_L128_496_views(cuda_device):
    w = synth.workloads.named("fp32_L128")
    proj = w.projections(device=cuda_device)
    host = proj.cpu().numpy()
    got = gpu_backproject(w, proj, tuning=tuning_mod.lookup(w.L, "f32", "soft"))
    ref = oracle_volume(w, host)
    assert_parity(got, ref, "L=128 x 496 full volume")


@pytest.mark.parametrize("name,dtype,frame", [("fp32_L512", "f32", "global"), ("fp32_L512", "f32", "block"),
                                              ("fp32_L1024", "f32", "global"), ("prec_L512", "f16", "global"),
                                              ("prec_L512", "bf16", "global"), ("fp32_L1024", "f16", "global")])
def test_sampled_parity_large(cuda_device, name, dtype, frame):
    w = synth.workloads.named(name)
    proj = w.projections(device=cuda_device)
    host = proj.cpu().numpy()
    tun = tuning_mod.lookup(w.L, dtype, "soft")
    stream = torch.cuda.current_stream()
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
        bp.set_precision(DTYPES[dtype][0], rct.RCT_INTERP_SOFT)
        bp.set_frame(rct.RCT_FRAME_BLOCK if frame == "block" else rct.RCT_FRAME_GLOBAL)
        bp.set_tuning(**tun)
        data = stored(proj, dtype)
        del proj
        bp.backproject(data, 0, w.n_views, stream)
        vol = torch.empty((w.L,) * 3, dtype=torch.float32, device=cuda_device)
        bp.read_volume(vol, stream)
        torch.cuda.synchronize()
    del data
    # L = 1024: 2^20 random voxels and two whole planes; smaller volumes: 2^15 and one plane
    idx = (_sample_indices(w.L, seed=w.seed, n_random=1 << 20, planes=(w.L // 4, (3 * w.L) // 4))
           if w.L >= 1024 else _sample_indices(w.L, seed=w.seed, planes=(w.L // 2,)))
    got = vol.view(-1)[torch.from_numpy(idx).to(cuda_device)].cpu().numpy()
    del vol
    ref = _sampled_reference(w, oracle_inputs(host, dtype), idx)
    # block frames keep every FP32 coordinate a short local offset: a ten times tighter bar
    tol = 1e-6 if frame == "block" else 1e-5
    assert_parity(got, ref, f"{name} {dtype} {frame} frame sampled ({idx.size} voxels)", rms_tol=tol)


def test_maximum_volume_L2048(cuda_device):
    """The largest volume the library accepts (2048^3 FP32 = 32 GiB), 64 full-size views (the FP32
    rounding noise of the coordinates averages over views; the bar is stated for full scans)."""
    w = synth.make_workload(2048, n_views=64, seed=1408)
    proj = w.projections(device=cuda_device)
    host = proj.cpu().numpy()
    tun = tuning_mod.lookup(w.L, "f32", "soft")
    stream = torch.cuda.current_stream()
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**tun)
        bp.backproject(proj, 0, w.n_views, stream)
        dev_vol = torch.empty((w.L,) * 3, dtype=torch.float32, device=cuda_device)
        bp.read_volume(dev_vol, stream)
        torch.cuda.synchronize()
    idx = _sample_indices(w.L, seed=w.seed, n_random=1 << 14, planes=(w.L // 2,))
    got = dev_vol.view(-1)[torch.from_numpy(idx).to(cuda_device)].cpu().numpy()
    del dev_vol
    ref = _sampled_reference(w, host, idx)
    assert_parity(got, ref, f"L=2048 sampled ({idx.size} voxels)")


def scaled_rms_tol(det_w: int, n_views: int) -> float:
    """The FP32 bar scaled off the stated configuration (1248-pixel rows, 496 views): the rounding error
    of an FP32 detector coordinate grows with its magnitude (proportional to the row length), and
    independent per-view errors shrink relative to the summed signal as 1/sqrt(views)."""
    return 1e-5 * max(1.0, det_w / 1248.0) * max(1.0, (496.0 / n_views) ** 0.5)


def test_large_detector(cuda_device):
    """A 4096 x 3072 detector (12.6 Mpx per view) through every gather route."""
    w = synth.make_workload(48, n_views=32, det_w=4096, det_h=3072, seed=1409)
    proj = w.projections(device=cuda_device)
    ref = oracle_volume(w, proj.cpu().numpy())
    tol = scaled_rms_tol(w.geom.det_w, w.n_views)
    for g in (rct.RCT_GATHER_TLD4, rct.RCT_GATHER_PAIR, rct.RCT_GATHER_QUAD, rct.RCT_GATHER_LDG):
        got = gpu_backproject(w, proj, tuning=dict(gather=g, views_per_pass=4))
        rms_g, _ = assert_parity(got, ref, f"4096x3072 detector, gather {g}", rms_tol=tol)
        # Block frames: here one voxel spans about 85 pixels, so a thread block's local offsets are
        # as long as the global ones and the frame brings nothing; the same scaled bar.
        got = gpu_backproject(w, proj, tuning=dict(gather=g, views_per_pass=4), frame=rct.RCT_FRAME_BLOCK)
        assert_parity(got, ref, f"4096x3072 detector, gather {g}, block frame", rms_tol=tol)


def test_sampled_truncating_rule_L512(cuda_device):
    """The RabbitCT cell rule at the benchmark's size and tuning, against the oracle run with the same
    rule on sampled voxels.  Truncation jumps where a detector coordinate crosses -1 or -2; a voxel
    within rounding of those points in some view has two valid results and is left out (FP64 test)."""
    w = synth.workloads.named("fp32_L512")
    proj = w.projections(device=cuda_device)
    host = proj.cpu().numpy()
    tun = tuning_mod.lookup(w.L, "f32", "soft")
    stream = torch.cuda.current_stream()
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**tun)
        bp.set_index_rule(rct.RCT_INDEX_TRUNC)
        bp.backproject(proj, 0, w.n_views, stream)
        vol = torch.empty((w.L,) * 3, dtype=torch.float32, device=cuda_device)
        bp.read_volume(vol, stream)
        torch.cuda.synchronize()
    del proj
    # sampled voxels: random ones, a plane at the volume's edge in z (projects above / below the detector
    # in part of the views) and the middle plane
    idx = _sample_indices(w.L, seed=w.seed + 1, planes=(0, w.L // 2))
    got = vol.view(-1)[torch.from_numpy(idx).to(cuda_device)].cpu().numpy()
    del vol
    L = w.L
    z, rem = np.divmod(idx, L * L)
    y, x = np.divmod(rem, L)
    P = np.stack([w.origin[0] + x * w.spacing[0], w.origin[1] + y * w.spacing[1], w.origin[2] + z * w.spacing[2],
                  np.ones(idx.size)])
    near = np.zeros(idx.size, dtype=bool)
    for A in np.asarray(w.geom.matrices, dtype=np.float64).reshape(-1, 3, 4):
        u, v, ww = A @ P
        for edge in (-1.0, -2.0):
            near |= (np.abs(u / ww - edge) < 2e-3) | (np.abs(v / ww - edge) < 2e-3)
    assert near.mean() < 0.01, near.mean()
    ref = oracle.backproject_voxels(w.L, w.geom.det_w, w.geom.det_h, w.geom.matrices, w.origin, w.spacing,
                                    host, idx, n_threads=oracle.max_threads(), index_rule=oracle.INDEX_TRUNC)
    assert_parity(got[~near], ref[~near], f"fp32_L512 truncating rule sampled ({int((~near).sum())} voxels)")
    floor_ref = _sampled_reference(w, host, idx)
    assert np.linalg.norm(floor_ref - ref) / np.linalg.norm(ref) > 1e-6      # the rule changes these sums


def test_parity_bar_scales_with_the_detector_width(cuda_device):
    """The scaled bar's premise, measured: with the field of view and the view count fixed, the FP32 error
    against the oracle grows with the detector's row length (an FP32 coordinate's rounding grows with its
    magnitude), and at each width it stays within the bar scaled by W / 1248 and sqrt(496 / views)."""
    errs = {}
    for det_w, det_h in [(1248, 960), (4096, 3151)]:
        w = synth.make_workload(48, n_views=32, det_w=det_w, det_h=det_h, seed=1411)
        proj = w.projections(device=cuda_device)
        got = gpu_backproject(w, proj, tuning=tuning_mod.lookup(512, "f32", "soft"))
        ref = oracle_volume(w, proj.cpu().numpy())
        del proj
        errs[det_w] = assert_parity(got, ref, f"{det_w}x{det_h}, 32 views",
                                    rms_tol=scaled_rms_tol(det_w, w.n_views))[0]
    assert errs[4096] > 1.5 * errs[1248], errs        # larger coordinates, larger rounding
