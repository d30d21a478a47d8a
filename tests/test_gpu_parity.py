"""CUDA path vs the FP64 oracle, element by element, through the C ABI (needs a GPU)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1401_7494_gb300 import rct
from gpu_helpers import (assert_parity, gpu_backproject, oracle_inputs, oracle_volume, rel_errors,
                         REL_RMS_TOL, MAX_ABS_TOL)

pytestmark = pytest.mark.gpu

# Small cases: several thread blocks and z-runs, ragged tails in x, y and z.
SMALL = {
    "L37": dict(L=37, n_views=20, det_w=96, det_h=74, seed=21),
    "L40": dict(L=40, n_views=33, det_w=130, det_h=100, seed=22),
    "L64": dict(L=64, n_views=40, det_w=160, det_h=123, seed=23),
}


def _case(name, device):
    w = synth.make_workload(**SMALL[name])
    proj = w.projections(device=device)
    return w, proj, proj.cpu().numpy()


@pytest.fixture(scope="module")
def small_cases(cuda_device):
    return {k: _case(k, cuda_device) for k in SMALL}


TUNINGS = [
    dict(gather=rct.RCT_GATHER_TLD4),
    dict(gather=rct.RCT_GATHER_LDG),
    dict(gather=rct.RCT_GATHER_TLD4, views_per_pass=7, zrun=8, xvec=1, block_x=64, block_y=2),
    dict(gather=rct.RCT_GATHER_LDG, views_per_pass=32, zrun=1, xvec=1, block_x=32, block_y=4),
    dict(gather=rct.RCT_GATHER_TLD4, views_per_pass=3, zrun=2, xvec=2, block_x=16, block_y=16),
    dict(gather=rct.RCT_GATHER_MIX, tex_zrun=2, views_per_pass=16, zrun=4, block_x=32, block_y=8),
    dict(gather=rct.RCT_GATHER_MIX, tex_zrun=5, views_per_pass=9, zrun=8, xvec=2, block_x=16, block_y=8),
    dict(gather=rct.RCT_GATHER_QUAD, views_per_pass=16, zrun=4, xvec=1, block_x=32, block_y=8),
    dict(gather=rct.RCT_GATHER_QUAD, views_per_pass=5, zrun=2, xvec=4, block_x=8, block_y=8),
    dict(gather=rct.RCT_GATHER_PAIR, views_per_pass=16, zrun=8, xvec=1, block_x=16, block_y=8),
    dict(gather=rct.RCT_GATHER_PAIR, views_per_pass=11, zrun=1, xvec=2, block_x=32, block_y=2),
    dict(gather=rct.RCT_GATHER_PAIR, views_per_pass=16, zrun=16, xvec=1, block_x=8, block_y=16),
    dict(gather=rct.RCT_GATHER_TLD4, views_per_pass=8, zrun=16, xvec=2, block_x=16, block_y=8),
    dict(gather=rct.RCT_GATHER_DQUAD, views_per_pass=24, zrun=8, xvec=1, block_x=8, block_y=16),
    dict(gather=rct.RCT_GATHER_DQUAD, views_per_pass=7, zrun=16, xvec=2, block_x=16, block_y=8),
    dict(gather=rct.RCT_GATHER_DQUAD, views_per_pass=13, zrun=2, xvec=4, block_x=8, block_y=8),
    dict(gather=rct.RCT_GATHER_LDG, views_per_pass=32, zrun=4, xvec=1, block_x=8, block_y=16, view_split=4),
    dict(gather=rct.RCT_GATHER_PAIR, views_per_pass=7, zrun=16, xvec=2, block_x=8, block_y=16, view_split=8),
    dict(gather=rct.RCT_GATHER_TLD4, views_per_pass=9, zrun=2, xvec=1, block_x=16, block_y=8, view_split=2),
]


@pytest.mark.parametrize("case", sorted(SMALL))
@pytest.mark.parametrize("ti", range(len(TUNINGS)))
def test_fp32_parity_small(small_cases, case, ti):
    w, proj, host = small_cases[case]
    tuning = dict(TUNINGS[ti])
    if w.L % tuning.get("xvec", 1):
        tuning["xvec"] = 1
    got = gpu_backproject(w, proj, tuning=tuning)
    ref = oracle_volume(w, host)
    assert_parity(got, ref, f"{case} tuning {tuning}")


@pytest.mark.parametrize("case", ["L40", "L64"])
def test_fp32_parity_xvec4(small_cases, case):
    w, proj, host = small_cases[case]
    got = gpu_backproject(w, proj, tuning=dict(xvec=4, block_x=8, block_y=8, zrun=4))
    assert_parity(got, oracle_volume(w, host), f"{case} xvec=4")


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
@pytest.mark.parametrize("gather", [rct.RCT_GATHER_TLD4, rct.RCT_GATHER_LDG, rct.RCT_GATHER_MIX,
                                    rct.RCT_GATHER_QUAD, rct.RCT_GATHER_PAIR])
def test_reduced_precision_storage_parity(small_cases, dtype, gather):
    """FP16/BF16 storage: same parity bar against the oracle fed the rounded projections."""
    w, proj, host = small_cases["L40"]
    got = gpu_backproject(w, proj, dtype=dtype, tuning=dict(gather=gather, tex_zrun=2, zrun=4))
    assert_parity(got, oracle_volume(w, oracle_inputs(host, dtype)), f"{dtype} storage")
    # and the stated (not gated) error against the FP32-input oracle stays small
    rms, _ = rel_errors(got, oracle_volume(w, host))
    assert rms < 5e-2 if dtype == "bf16" else rms < 5e-3


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_texture_interp_error_is_bounded(small_cases, dtype):
    """Hardware bilinear uses fixed-point weights: its error is reported, with a loose sanity bound."""
    w, proj, host = small_cases["L64"]
    got = gpu_backproject(w, proj, dtype=dtype, interp=rct.RCT_INTERP_TEX)
    rms, mx = rel_errors(got, oracle_volume(w, oracle_inputs(host, dtype)))
    assert rms < 2e-2 and mx < 5e-2, (rms, mx)


def test_convert_projections_bit_exact(cuda_device):
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(size=100003) * 10.0 ** rng.uniform(-6, 5, size=100003),
                        [0.0, -0.0, 65504.0, 65520.0, 1e-8, 3.3895e38]]).astype(np.float32)
    src = torch.from_numpy(x).to(cuda_device)
    for name, code, tdt, ref in [("f16", rct.RCT_PROJ_F16, torch.float16, oracle.round_f16),
                                 ("bf16", rct.RCT_PROJ_BF16, torch.bfloat16, oracle.round_bf16)]:
        dst = torch.empty(x.size, dtype=tdt, device=cuda_device)
        rct.rct_convert_projections(src, dst, x.size, code, torch.cuda.current_stream())
        got = dst.float().cpu().numpy()
        exp = ref(x)
        assert np.array_equal(got, exp, equal_nan=True), name


def test_views_per_pass_does_not_change_bits(small_cases):
    """The per-voxel sum runs in view order whatever K is; partial sums round-trip through FP32 exactly."""
    w, proj, _ = small_cases["L37"]
    vols = [gpu_backproject(w, proj, tuning=dict(views_per_pass=k, zrun=4, xvec=1, gather=rct.RCT_GATHER_TLD4))
            for k in (1, 5, 32)]
    assert np.array_equal(vols[0], vols[1]) and np.array_equal(vols[0], vols[2])


def test_split_calls_and_checkpoint_resume(small_cases, cuda_device):
    w, proj, _ = small_cases["L37"]
    tun = dict(views_per_pass=4, zrun=2, gather=rct.RCT_GATHER_LDG)
    whole = gpu_backproject(w, proj, tuning=tun)
    # split at a batch boundary: identical bits
    split = gpu_backproject(w, proj, tuning=tun, chunks=[(0, 8), (8, w.n_views)])
    assert np.array_equal(whole, split)
    # checkpoint after 8 views, restore into a fresh context, continue
    stream = torch.cuda.current_stream()
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as a:
        a.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**tun)
        a.backproject(proj[:8], 0, 8, stream)
        ckpt = torch.empty((w.L,) * 3, device=cuda_device)
        a.read_volume(ckpt, stream)
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as b:
        b.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**tun)
        b.write_volume(ckpt, stream)
        b.backproject(proj[8:], 8, w.n_views - 8, stream)
        out = torch.empty_like(ckpt)
        b.read_volume(out, stream)
        torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), whole)


def test_host_input_path_matches_device_path(small_cases):
    """The host-input path (batched uploads and staging on the copy stream) gives the device path's volume bit
    for bit, for every gather route and a ragged last batch."""
    w, proj, host = small_cases["L40"]
    for gather, K in ((rct.RCT_GATHER_TLD4, 5), (rct.RCT_GATHER_LDG, 5), (rct.RCT_GATHER_MIX, 5),
                      (rct.RCT_GATHER_QUAD, 5), (rct.RCT_GATHER_PAIR, 5), (rct.RCT_GATHER_PAIR, 24),
                      (rct.RCT_GATHER_DQUAD, 16)):
        tun = dict(views_per_pass=K, gather=gather, zrun=4, tex_zrun=1)
        dev = gpu_backproject(w, proj, tuning=tun)
        pinned = torch.from_numpy(host).pin_memory()
        stream = torch.cuda.current_stream()
        with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
            bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**tun)
            bp.backproject_host(pinned, 0, w.n_views, stream)
            out = np.empty((w.L,) * 3, np.float32)
            torch.cuda.synchronize()
            bp.read_volume(out, stream)
            torch.cuda.synchronize()
        assert np.array_equal(out, dev), f"gather {gather}, K={K}"


def test_reset_and_zero_volume(small_cases, cuda_device):
    w, proj, _ = small_cases["L37"]
    stream = torch.cuda.current_stream()
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
        out = torch.full((w.L,) * 3, 7.0, device=cuda_device)
        bp.read_volume(out, stream)                  # fresh context reads zeros
        torch.cuda.synchronize()
        assert float(out.abs().max()) == 0.0
        bp.backproject(proj, 0, w.n_views, stream)
        first = torch.empty_like(out)
        bp.read_volume(first, stream)
        bp.reset(stream)
        bp.backproject(proj, 0, w.n_views, stream)   # after reset: same as fresh
        second = torch.empty_like(out)
        bp.read_volume(second, stream)
        bp.backproject(proj[:0], 0, 0, stream)        # n == 0 is a no-op
        torch.cuda.synchronize()
        assert torch.equal(first, second)
        assert bp.launches > 0


def test_argument_errors(cuda_device):
    w = synth.make_workload(8, n_views=4, det_w=16, det_h=12, seed=1)
    proj = torch.zeros((4, 12, 16), device=cuda_device)
    with rct.Backprojector(8, 16, 12, 4) as bp:
        with pytest.raises(rct.RctError) as e:
            bp.backproject(proj, 0, 4)
        assert e.value.status == rct.RCT_ESTATE
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
        for first, n in [(-1, 2), (3, 2), (0, -1)]:
            with pytest.raises(rct.RctError) as e:
                rct.rct_backproject(bp.ctx, proj, first, n, None)
            assert e.value.status == rct.RCT_EINVAL
        with pytest.raises(rct.RctError):
            rct.rct_backproject(bp.ctx, 0, 0, 2, None)
        for bad in [dict(views_per_pass=33), dict(zrun=3), dict(zrun=16, xvec=4), dict(xvec=3), dict(block_x=7, block_y=1),
                    dict(block_x=1024, block_y=1), dict(gather=9), dict(gather=7), dict(tex_zrun=17)]:
            with pytest.raises(rct.RctError):
                bp.set_tuning(**bad)
        with pytest.raises(rct.RctError):
            bp.set_precision(5, 0)
    with pytest.raises(rct.RctError):
        rct.rct_create(0, 16, 16, 4)


def test_degenerate_volumes(cuda_device):
    """L = 1 and L = 2 (smaller than every tile), and a volume entirely off the detector."""
    for L in (1, 2, 3):
        w = synth.make_workload(L, n_views=9, det_w=40, det_h=30, seed=30 + L)
        proj = w.projections(device=cuda_device)
        got = gpu_backproject(w, proj, tuning=dict(zrun=8, views_per_pass=4))
        assert_parity(got, oracle_volume(w, proj.cpu().numpy()), f"L={L}")
    w = synth.make_workload(12, n_views=5, det_w=40, det_h=30, seed=40)
    w.origin = w.origin + np.array([0.0, 0.0, 5000.0])     # far above the field of view, still w > 0
    proj = w.projections(device=cuda_device)
    got = gpu_backproject(w, proj)
    ref = oracle_volume(w, proj.cpu().numpy())
    assert np.all(got == 0.0) and np.all(ref == 0.0)


def test_all_gather_routes_agree_closely(small_cases):
    """Texture gather, plain loads and quad loads fetch the same taps; only the lerp's rounding differs."""
    w, proj, _ = small_cases["L64"]
    vols = {g: gpu_backproject(w, proj, tuning=dict(gather=g, zrun=4, xvec=1, views_per_pass=16))
            for g in (rct.RCT_GATHER_TLD4, rct.RCT_GATHER_LDG, rct.RCT_GATHER_QUAD, rct.RCT_GATHER_PAIR)}
    ref = vols[rct.RCT_GATHER_LDG].astype(np.float64)
    for g, v in vols.items():
        rms, mx = rel_errors(v, ref)
        assert rms < 1e-6 and mx < 1e-5, (g, rms, mx)


# Block frames (rct_set_frame): the same parity bar on the small cases (their volumes span only a
# few thread blocks, so the frame's gain shows at L = 512, tested with the sampled configurations).
@pytest.mark.parametrize("case", sorted(SMALL))
@pytest.mark.parametrize("ti", [1, 3, 4, 5, 7, 8, 9, 11, 12])
def test_block_frame_parity_small(small_cases, case, ti):
    w, proj, host = small_cases[case]
    tuning = dict(TUNINGS[ti])
    if w.L % tuning.get("xvec", 1):
        tuning["xvec"] = 1
    got = gpu_backproject(w, proj, tuning=tuning, frame=rct.RCT_FRAME_BLOCK)
    assert_parity(got, oracle_volume(w, host), f"{case} block frame, tuning {tuning}")


def test_block_frame_routes_agree(small_cases):
    """With block frames too, every gather route fetches the same taps."""
    w, proj, _ = small_cases["L64"]
    vols = {g: gpu_backproject(w, proj, tuning=dict(gather=g, zrun=4, xvec=1, views_per_pass=16),
                               frame=rct.RCT_FRAME_BLOCK)
            for g in (rct.RCT_GATHER_TLD4, rct.RCT_GATHER_LDG, rct.RCT_GATHER_QUAD, rct.RCT_GATHER_PAIR)}
    ref = vols[rct.RCT_GATHER_LDG].astype(np.float64)
    for g, v in vols.items():
        rms, mx = rel_errors(v, ref)
        assert rms < 1e-6 and mx < 1e-5, (g, rms, mx)


def test_frame_argument_errors(cuda_device):
    with rct.Backprojector(8, 16, 12, 4) as bp:
        assert rct.rct_get_frame(bp.ctx) == rct.RCT_FRAME_GLOBAL
        for bad in (-1, 2):
            with pytest.raises(rct.RctError) as e:
                bp.set_frame(bad)
            assert e.value.status == rct.RCT_EINVAL
        bp.set_frame(rct.RCT_FRAME_BLOCK)
        assert rct.rct_get_frame(bp.ctx) == rct.RCT_FRAME_BLOCK
        for dtype, interp in ((rct.RCT_PROJ_F16, rct.RCT_INTERP_SOFT), (rct.RCT_PROJ_BF16, rct.RCT_INTERP_SOFT),
                              (rct.RCT_PROJ_F32, rct.RCT_INTERP_TEX)):
            with pytest.raises(rct.RctError) as e:
                bp.set_precision(dtype, interp)
            assert e.value.status == rct.RCT_ENOTSUP
        bp.set_frame(rct.RCT_FRAME_GLOBAL)
        bp.set_precision(rct.RCT_PROJ_F16, rct.RCT_INTERP_SOFT)
        with pytest.raises(rct.RctError) as e:
            bp.set_frame(rct.RCT_FRAME_BLOCK)
        assert e.value.status == rct.RCT_ENOTSUP
        assert rct.rct_get_frame(bp.ctx) == rct.RCT_FRAME_GLOBAL


def _near_trunc_edge(w, tol_px):
    """(L, L, L) mask of voxels whose detector coordinate lies within tol_px of -1 or -2 in some view (FP64)."""
    L = w.L
    ax = [w.origin[k] + np.arange(L) * w.spacing[k] for k in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    P = np.stack([x.ravel(), y.ravel(), z.ravel(), np.ones(L ** 3)])
    near = np.zeros(L ** 3, dtype=bool)
    for A in np.asarray(w.geom.matrices, dtype=np.float64).reshape(-1, 3, 4):
        u, v, ww = A @ P
        for edge in (-1.0, -2.0):
            near |= (np.abs(u / ww - edge) < tol_px) | (np.abs(v / ww - edge) < tol_px)
    return near.reshape(L, L, L)


# RabbitCT compatibility: Listing 1's truncating cell index, against the oracle run with the same rule.
@pytest.mark.parametrize("case", sorted(SMALL))
@pytest.mark.parametrize("tuning", [dict(), dict(zrun=8, xvec=1, block_x=16, block_y=8, views_per_pass=16),
                                    dict(zrun=2, xvec=2, block_x=32, block_y=4, views_per_pass=7),
                                    dict(gather=rct.RCT_GATHER_PAIR, zrun=4, views_per_pass=16)])
def test_truncating_index_parity(small_cases, case, tuning):
    w, proj, host = small_cases[case]
    tuning = dict(tuning)
    if w.L % tuning.get("xvec", 1):
        tuning["xvec"] = 1
    got = gpu_backproject(w, proj, tuning=tuning, index_rule=rct.RCT_INDEX_TRUNC)
    ref = oracle_volume(w, host, index_rule=oracle.INDEX_TRUNC)
    # Truncation jumps at coordinates -1 and -2 (just right of -1 the cell extrapolates from the two
    # edge taps; just right of -2 tap 0 carries weight -1; at either point the value is 0), so a voxel
    # within rounding of those edges in some view has two valid results; compare the others element
    # by element.
    ambiguous = _near_trunc_edge(w, 2e-3)
    assert ambiguous.mean() < 0.01, ambiguous.mean()
    assert_parity(got[~ambiguous], ref[~ambiguous], f"{case} truncating index, tuning {tuning}")
    # the rule matters on these cases: voxels project into the band left of / above the detector
    floor_ref = oracle_volume(w, host)
    assert rel_errors(floor_ref, ref)[0] > 1e-4


def test_rabbitct_geometry_setter(small_cases, cuda_device):
    """Column-major FP32 matrices with scalar O / MM give the same volume as the same values passed
    row-major in FP64 with per-axis origin and spacing."""
    w, proj, _ = small_cases["L40"]
    A = np.asarray(w.geom.matrices, dtype=np.float32)                 # (n, 3, 4) rounded to FP32
    colmajor = np.ascontiguousarray(np.transpose(A.reshape(-1, 3, 4), (0, 2, 1)))   # element (r, c) at [c, r]
    O, MM = np.float32(w.origin[0]), np.float32(w.spacing[0])
    assert np.allclose(w.origin, w.origin[0]) and np.allclose(w.spacing, w.spacing[0])
    stream = torch.cuda.current_stream()
    vols = []
    for mode in ("rabbitct", "rowmajor"):
        with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
            if mode == "rabbitct":
                rct.rct_set_geometry_rabbitct(bp.ctx, colmajor, float(O), float(MM))
            else:
                bp.set_geometry(A.astype(np.float64), np.full(3, float(O)), np.full(3, float(MM)))
            bp.set_index_rule(rct.RCT_INDEX_TRUNC)
            bp.backproject(proj, 0, w.n_views, stream)
            out = torch.empty((w.L,) * 3, dtype=torch.float32, device=cuda_device)
            bp.read_volume(out, stream)
            torch.cuda.synchronize()
            vols.append(out.cpu().numpy())
    assert np.array_equal(vols[0], vols[1])


def test_index_rule_argument_errors(cuda_device):
    with rct.Backprojector(8, 16, 12, 4) as bp:
        assert rct.rct_get_index_rule(bp.ctx) == rct.RCT_INDEX_FLOOR
        for bad in (-1, 2):
            with pytest.raises(rct.RctError) as e:
                bp.set_index_rule(bad)
            assert e.value.status == rct.RCT_EINVAL
        bp.set_index_rule(rct.RCT_INDEX_TRUNC)
        assert rct.rct_get_index_rule(bp.ctx) == rct.RCT_INDEX_TRUNC
        for dtype, interp in ((rct.RCT_PROJ_F16, rct.RCT_INTERP_SOFT), (rct.RCT_PROJ_F32, rct.RCT_INTERP_TEX)):
            with pytest.raises(rct.RctError) as e:
                bp.set_precision(dtype, interp)
            assert e.value.status == rct.RCT_ENOTSUP
        with pytest.raises(rct.RctError) as e:
            bp.set_frame(rct.RCT_FRAME_BLOCK)
        assert e.value.status == rct.RCT_ENOTSUP
        bp.set_index_rule(rct.RCT_INDEX_FLOOR)
        bp.set_frame(rct.RCT_FRAME_BLOCK)
        with pytest.raises(rct.RctError) as e:
            bp.set_index_rule(rct.RCT_INDEX_TRUNC)
        assert e.value.status == rct.RCT_ENOTSUP
        with pytest.raises(rct.RctError) as e:
            rct.rct_set_geometry_rabbitct(bp.ctx, np.zeros(12 * 4, np.float32), 0.0, -1.0)   # spacing <= 0
        assert e.value.status == rct.RCT_EINVAL


@pytest.mark.parametrize("case", ["L37", "L64"])
@pytest.mark.parametrize("tuning,frame", [(dict(zrun=8, views_per_pass=16), rct.RCT_FRAME_GLOBAL),
                                          (dict(zrun=4, views_per_pass=7, gather=rct.RCT_GATHER_PAIR), rct.RCT_FRAME_GLOBAL),
                                          (dict(zrun=2, xvec=1, views_per_pass=32), rct.RCT_FRAME_BLOCK),
                                          (dict(zrun=16, xvec=1, gather=rct.RCT_GATHER_TLD4), rct.RCT_FRAME_GLOBAL)])
def test_overlapped_read_back_is_bitwise_the_separate_calls(small_cases, cuda_device, case, tuning, frame):
    """rct_backproject_host_read (last pass in z-slabs, each copied out when done) against
    rct_backproject_host + rct_read_volume: same bits, to pinned host memory and to device memory, also
    after an earlier call has filled part of the volume."""
    w, proj, _ = small_cases[case]
    pinned = proj.cpu().pin_memory()
    stream = torch.cuda.current_stream()
    split = w.n_views // 3
    shape = (w.L,) * 3
    outs = {}
    for mode in ("separate", "host", "device"):
        with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
            bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_frame(frame).set_tuning(**tuning)
            bp.backproject_host(pinned[:split], 0, split, stream)
            rest = pinned[split:]
            if mode == "separate":
                dst = torch.empty(shape, dtype=torch.float32, device=cuda_device)
                bp.backproject_host(rest, split, w.n_views - split, stream)
                bp.read_volume(dst, stream)
            elif mode == "host":
                dst = torch.empty(shape, dtype=torch.float32).pin_memory()
                bp.backproject_host_read(rest, dst, split, w.n_views - split, stream)
            else:
                dst = torch.empty(shape, dtype=torch.float32, device=cuda_device)
                bp.backproject_host_read(rest, dst, split, w.n_views - split, stream)
            stream.synchronize()
            outs[mode] = dst.cpu()
    assert torch.equal(outs["host"], outs["separate"])
    assert torch.equal(outs["device"], outs["separate"])


def test_overlapped_read_back_edge_cases(small_cases, cuda_device):
    w, proj, host = small_cases["L40"]
    pinned = proj.cpu().pin_memory()
    stream = torch.cuda.current_stream()
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
        dst = torch.full((w.L,) * 3, 7.0).pin_memory()
        bp.backproject_host_read(pinned[:0], dst, 0, 0, stream)           # n == 0: the (zero) volume
        stream.synchronize()
        assert torch.count_nonzero(dst) == 0
        bp.backproject_host_read(pinned, dst, 0, w.n_views, stream)        # one call, whole scan
        stream.synchronize()
        assert_parity(dst.numpy(), oracle_volume(w, host), "overlapped read-back")
        with pytest.raises(rct.RctError) as e:
            rct.rct_backproject_host_read(bp.ctx, pinned, 0, 1, 0, None)
        assert e.value.status == rct.RCT_EINVAL


def test_graph_refuses_to_launch_after_its_state_is_replaced(small_cases, cuda_device):
    """A captured pass replays the direct call bit for bit; once its context reallocates the staging the
    graph points at (a larger K), takes a new geometry, or is destroyed, launching it is RCT_ESTATE and
    runs nothing."""
    w, proj, _ = small_cases["L37"]
    tun = dict(views_per_pass=4, zrun=4, gather=rct.RCT_GATHER_PAIR)
    direct = gpu_backproject(w, proj, tuning=tun)
    stream = torch.cuda.Stream(device=cuda_device)
    out = torch.empty((w.L,) * 3, device=cuda_device)

    def capture(bp):
        rct.rct_prepare(bp.ctx, False)
        bp.reset(stream)
        rct.rct_graph_begin(stream)
        try:
            bp.backproject(proj, 0, w.n_views, stream)
        finally:
            g = rct.rct_graph_end(stream)
        return g

    for change in ("larger_k", "geometry", "destroyed"):
        bp = rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views)
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**tun)
        g = capture(bp)
        try:
            rct.rct_graph_launch(g, stream)
            bp.read_volume(out, stream)
            stream.synchronize()
            assert np.array_equal(out.cpu().numpy(), direct)
            if change == "larger_k":
                bp.set_tuning(**dict(tun, views_per_pass=8))
                bp.backproject(proj, 0, w.n_views, stream)      # reallocates the pair staging
            elif change == "geometry":
                bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
            else:
                bp.close()
            with pytest.raises(rct.RctError) as e:
                rct.rct_graph_launch(g, stream)
            assert e.value.status == rct.RCT_ESTATE
            stream.synchronize()
        finally:
            rct.rct_graph_destroy(g)
            bp.close()
    # a smaller K reuses the staging: the graph stays valid
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**tun)
        g = capture(bp)
        try:
            bp.set_tuning(**dict(tun, views_per_pass=2))
            bp.backproject(proj, 0, w.n_views, stream)
            rct.rct_graph_launch(g, stream)
            bp.read_volume(out, stream)
            stream.synchronize()
            assert np.array_equal(out.cpu().numpy(), direct)
        finally:
            rct.rct_graph_destroy(g)


def test_graph_replay_of_the_host_input_step_is_bitwise_the_direct_call(small_cases, cuda_device):
    """The host-input step with the overlapped read-back (copy stream, staging kernels at high priority, z-slab
    read-back) captured into a graph and replayed writes the same bits as the direct call."""
    w, proj, host = small_cases["L40"]
    pinned = torch.from_numpy(host).pin_memory()
    stream = torch.cuda.Stream(device=cuda_device)
    for tun in (dict(gather=rct.RCT_GATHER_PAIR, views_per_pass=5, zrun=4),
                dict(gather=rct.RCT_GATHER_TLD4, views_per_pass=7, zrun=8)):
        with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
            bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**tun)
            direct = torch.empty((w.L,) * 3, dtype=torch.float32).pin_memory()
            bp.reset(stream)
            bp.backproject_host_read(pinned, direct, 0, w.n_views, stream)
            stream.synchronize()
            replayed = torch.zeros_like(direct).pin_memory()
            bp.reset(stream)
            rct.rct_graph_begin(stream)
            try:
                bp.backproject_host_read(pinned, replayed, 0, w.n_views, stream)
            finally:
                g = rct.rct_graph_end(stream)
            try:
                for _ in range(2):
                    replayed.zero_()
                    rct.rct_graph_launch(g, stream)
                    stream.synchronize()
                    assert torch.equal(replayed, direct), tun
            finally:
                rct.rct_graph_destroy(g)


@pytest.mark.parametrize("zrun,xvec", [(8, 1), (16, 2), (1, 4)])
def test_staged_routes_are_bitwise_equal(small_cases, zrun, xvec):
    """Quads, pairs and difference quads feed the same roundings to the same sums, on the fast path
    (warps wholly on the image) and off it: their volumes are identical, and so are the plain loads'."""
    w, proj, host = small_cases["L64"]
    base = dict(views_per_pass=12, zrun=zrun, xvec=xvec, block_x=8, block_y=16)
    vols = {g: gpu_backproject(w, proj, tuning=dict(base, gather=g))
            for g in (rct.RCT_GATHER_PAIR, rct.RCT_GATHER_QUAD, rct.RCT_GATHER_DQUAD, rct.RCT_GATHER_LDG)}
    ref = vols[rct.RCT_GATHER_PAIR]
    for g, v in vols.items():
        assert np.array_equal(v, ref), f"gather {g} differs from pairs"
    assert_parity(ref, oracle_volume(w, host), f"staged routes z-run {zrun} x-vector {xvec}")


def test_difference_quads_need_fp32(small_cases):
    w, proj, _ = small_cases["L37"]
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
        bp.set_precision(rct.RCT_PROJ_F16).set_tuning(gather=rct.RCT_GATHER_DQUAD)
        data = torch.empty(proj.shape, dtype=torch.float16, device=proj.device)
        with pytest.raises(rct.RctError) as e:
            bp.backproject(data, 0, w.n_views)
        assert e.value.status == rct.RCT_ENOTSUP


@pytest.mark.parametrize("split", [2, 4, 8])
def test_view_split_is_deterministic_and_close_to_the_plain_order(small_cases, cuda_device, split):
    """The view split regroups each voxel's sum (its groups' partial volumes are added after the call): two runs
    give the same bits, split calls and the host path with the overlapped read-back agree with the oracle, and
    the plain order is within rounding."""
    w, proj, host = small_cases["L40"]
    t = dict(gather=rct.RCT_GATHER_LDG, views_per_pass=11, zrun=4, xvec=1, block_x=8, block_y=16)
    plain = gpu_backproject(w, proj, tuning=t)
    a = gpu_backproject(w, proj, tuning=dict(t, view_split=split))
    b = gpu_backproject(w, proj, tuning=dict(t, view_split=split))
    assert np.array_equal(a, b)
    ref = oracle_volume(w, host)
    assert_parity(a, ref, f"view split {split}")
    assert rel_errors(a, plain)[0] < 1e-6
    chunks = gpu_backproject(w, proj, tuning=dict(t, view_split=split), chunks=[(0, 5), (5, 18), (18, w.n_views)])
    assert_parity(chunks, ref, f"view split {split}, three calls")
    stream = torch.cuda.current_stream()
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(**dict(t, view_split=split))
        out = torch.empty((w.L,) * 3, dtype=torch.float32, pin_memory=True)
        bp.backproject_host_read(proj.cpu().pin_memory(), out, 0, w.n_views, stream)
        torch.cuda.synchronize()
        assert np.array_equal(out.numpy(), a)                 # same passes, same groups: same bits


def test_view_split_needs_the_global_frame(small_cases):
    w, proj, _ = small_cases["L37"]
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing).set_tuning(view_split=4)
        bp.set_frame(rct.RCT_FRAME_BLOCK)
        with pytest.raises(rct.RctError) as e:
            bp.backproject(proj, 0, w.n_views)
        assert e.value.status == rct.RCT_ENOTSUP
        with pytest.raises(rct.RctError):
            bp.set_tuning(view_split=3)


@pytest.mark.parametrize("gather", [rct.RCT_GATHER_PAIR, rct.RCT_GATHER_TLD4, rct.RCT_GATHER_LDG])
def test_lane_map_does_not_change_bits(small_cases, gather):
    """Blocks 8 threads wide hand each half warp a 4 x 4 patch of voxel columns (fewer cache lines per 8-byte
    load); other widths keep the row order.  Which lane computes a voxel must not change its sum: in the global
    frame the volumes of 8 x 16 and 8 x 8 blocks (lane map) equal those of 16 x 8 and 32 x 4 blocks bit for bit,
    with ragged tails in x, y and z (L = 40)."""
    w, proj, host = small_cases["L40"]
    base = dict(gather=gather, views_per_pass=11, zrun=4, xvec=1)
    vols = {(bx, by): gpu_backproject(w, proj, tuning=dict(base, block_x=bx, block_y=by))
            for bx, by in [(8, 16), (8, 8), (16, 8), (32, 4)]}
    ref = vols[(16, 8)]
    for shape, v in vols.items():
        assert np.array_equal(v, ref), f"block {shape} differs from 16 x 8"
    assert_parity(ref, oracle_volume(w, host), f"lane map, gather {gather}")
