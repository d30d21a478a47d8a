"""Device pre-processing (cosine weight + ramp filter, rct_filter_projections) against the FP64
oracle, element by element, through the C ABI (needs a GPU)."""
import numpy as np
import pytest
import torch

import synth
from oracle import filter as of
from paper_1401_7494_gb300 import rct
from gpu_helpers import assert_parity, rel_errors

pytestmark = pytest.mark.gpu

CASES = {
    # ragged: odd row count (the last block filters one row), widths that are not powers of two
    "small": dict(L=16, n_views=6, det_w=97, det_h=33, seed=31),
    "mid": dict(L=16, n_views=4, det_w=300, det_h=21, seed=32),
    "full": dict(L=16, n_views=3, det_w=1248, det_h=960, seed=33),
}


def _raw(name, device):
    w = synth.make_workload(**CASES[name])
    raw = synth.make_projections(w.geom, w.phantom, device=device, weighted=False, filtered=False)
    return w, raw


def _filtered(w, raw, out_dtype=rct.RCT_PROJ_F32, in_place=False, first=0, n=None):
    n = w.n_views if n is None else n
    tdt = {rct.RCT_PROJ_F32: torch.float32, rct.RCT_PROJ_F16: torch.float16, rct.RCT_PROJ_BF16: torch.bfloat16}
    src = raw[first:first + n].clone()
    out = src if in_place else torch.empty(src.shape, dtype=tdt[out_dtype], device=raw.device)
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_filter(w.geom.sdd, w.geom.pitch, w.geom.principal)
        bp.filter(src, out, out_dtype, first, n, torch.cuda.current_stream())
        torch.cuda.synchronize()
    return out


def fp32_filter_tolerance(weighted: np.ndarray, ref: np.ndarray, W: int, pitch: float) -> float:
    """Relative-RMS bar for an FP32 transform-based ramp filter, from the arithmetic: each of the
    log2(N) passes of a length-N transform rounds with relative error 2^-24 in the 2-norm, and the
    filter scales that error by at most its largest spectral gain while the signal passes with the
    gain ||y|| / ||x'||, which is small: the ramp suppresses the rows' large low frequencies.  So
    rel-RMS <= 2^-24 * log2(N) * max|G| * ||x'|| / ||y||, with G the spectrum of tau * h."""
    N = 1 << int(np.ceil(np.log2(2 * W - 1)))
    n = np.arange(W, dtype=np.float64)
    h = -2.0 / (np.pi ** 2 * pitch ** 2 * (4.0 * n * n - 1.0))
    hp = np.zeros(N)
    hp[:W] = h
    hp[N - W + 1:] = h[1:][::-1]
    gain = np.max(np.abs(np.fft.fft(hp).real)) * pitch
    return 2.0 ** -24 * np.log2(N) * gain * np.linalg.norm(weighted) / np.linalg.norm(ref)


@pytest.mark.parametrize("name", sorted(CASES))
def test_filter_parity(cuda_device, name):
    w, raw = _raw(name, cuda_device)
    got = _filtered(w, raw).cpu().numpy()
    host = raw.cpu().numpy().astype(np.float64)
    ref = of.preprocess(host, w.geom.sdd, w.geom.pitch, w.geom.principal)
    weighted = np.stack([host[v] * of.cosine_weight(w.geom.det_w, w.geom.det_h, w.geom.sdd, w.geom.pitch,
                                                    *w.geom.principal[v]) for v in range(w.n_views)])
    tol = max(1e-5, fp32_filter_tolerance(weighted, ref, w.geom.det_w, w.geom.pitch))
    assert tol < 2e-4, tol
    assert_parity(got, ref, f"filter {name}", rms_tol=tol)


def test_filter_in_place_and_view_offsets(cuda_device):
    w, raw = _raw("mid", cuda_device)
    whole = _filtered(w, raw)
    assert torch.equal(_filtered(w, raw, in_place=True), whole)
    assert torch.equal(_filtered(w, raw, first=1, n=2), whole[1:3])      # principal points follow the view


@pytest.mark.parametrize("dtype,torch_dtype", [(rct.RCT_PROJ_F16, torch.float16), (rct.RCT_PROJ_BF16, torch.bfloat16)])
def test_filter_fused_narrowing_is_the_conversion(cuda_device, dtype, torch_dtype):
    """The 16-bit output equals the FP32 output converted by rct_convert_projections, bit for bit."""
    w, raw = _raw("small", cuda_device)
    f32 = _filtered(w, raw)
    fused = _filtered(w, raw, out_dtype=dtype)
    conv = torch.empty(f32.shape, dtype=torch_dtype, device=cuda_device)
    rct.rct_convert_projections(f32, conv, f32.numel(), dtype, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.equal(fused.view(torch.int16), conv.view(torch.int16))


def test_filter_matches_the_generators_fft_filter(cuda_device):
    """Consistency with the input generator's own pre-processing (an FP64 FFT in torch): the
    backprojection inputs of the benchmark are that generator's output."""
    w, raw = _raw("mid", cuda_device)
    got = _filtered(w, raw).cpu().numpy()
    gen = synth.make_projections(w.geom, w.phantom, device=cuda_device).cpu().numpy()
    rms, mx = rel_errors(got, gen)
    assert rms < 1e-4 and mx < 1e-4, (rms, mx)


def test_filter_argument_errors(cuda_device):
    w, raw = _raw("small", cuda_device)
    out16 = torch.empty(raw.shape, dtype=torch.float16, device=cuda_device)
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        with pytest.raises(rct.RctError) as e:
            bp.filter(raw, raw)
        assert e.value.status == rct.RCT_ESTATE
        for sdd, pitch in [(0.0, 0.3), (1200.0, -1.0), (float("nan"), 0.3)]:
            with pytest.raises(rct.RctError) as e:
                bp.set_filter(sdd, pitch, w.geom.principal)
            assert e.value.status == rct.RCT_EINVAL
        bp.set_filter(w.geom.sdd, w.geom.pitch, w.geom.principal)
        with pytest.raises(ValueError):                              # the binding checks a tensor's type
            rct.rct_filter_projections(bp.ctx, raw, raw, rct.RCT_PROJ_F16, 0, w.n_views, None)
        with pytest.raises(rct.RctError) as e:                       # 16-bit output over its own input
            rct.rct_filter_projections(bp.ctx, raw.data_ptr(), raw.data_ptr(), rct.RCT_PROJ_F16, 0, w.n_views, None)
        assert e.value.status == rct.RCT_EINVAL
        with pytest.raises(rct.RctError) as e:                       # partial overlap
            rct.rct_filter_projections(bp.ctx, raw, raw[1:], rct.RCT_PROJ_F32, 0, 2, None)
        assert e.value.status == rct.RCT_EINVAL
        for first, n in [(-1, 1), (w.n_views, 1), (0, -1)]:
            with pytest.raises(rct.RctError) as e:
                rct.rct_filter_projections(bp.ctx, raw, out16, rct.RCT_PROJ_F16, first, n, None)
            assert e.value.status == rct.RCT_EINVAL
        with pytest.raises(rct.RctError) as e:
            rct.rct_filter_projections(bp.ctx, raw, out16, 7, 0, 1, None)
        assert e.value.status == rct.RCT_EINVAL
        rct.rct_filter_projections(bp.ctx, raw, out16, rct.RCT_PROJ_F16, 0, 0, None)   # n == 0: no-op
    with rct.Backprojector(8, 9000, 4, 2) as bp:
        with pytest.raises(rct.RctError) as e:
            bp.set_filter(1200.0, 0.1, np.zeros((2, 2)))
        assert e.value.status == rct.RCT_ENOTSUP
