"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and compare with the oracle."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import synth
from paper_1401_7494_gb300 import rct

# Parity bar for the FP32 software-interpolated path (and for the reduced-precision
# storage variants against the oracle run on the same rounded projections).
REL_RMS_TOL = 1e-5
MAX_ABS_TOL = 1e-3          # times max |f_oracle|; covers floor() flips at pixel edges


def rel_errors(gpu: np.ndarray, ref: np.ndarray):
    g = np.asarray(gpu, np.float64).ravel()
    r = np.asarray(ref, np.float64).ravel()
    rms = float(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300))
    mx = float(np.max(np.abs(g - r)) / max(np.max(np.abs(r)), 1e-300)) if r.size else 0.0
    return rms, mx


def assert_parity(gpu, ref, what="", rms_tol=REL_RMS_TOL, max_tol=MAX_ABS_TOL):
    rms, mx = rel_errors(gpu, ref)
    assert rms <= rms_tol and mx <= max_tol, f"{what}: rel-RMS {rms:.3e} (tol {rms_tol:.0e}), max {mx:.3e} (tol {max_tol:.0e})"
    return rms, mx


DTYPES = {"f32": (rct.RCT_PROJ_F32, torch.float32), "f16": (rct.RCT_PROJ_F16, torch.float16),
          "bf16": (rct.RCT_PROJ_BF16, torch.bfloat16)}


def stored(proj_f32: torch.Tensor, dtype: str) -> torch.Tensor:
    """Projections in the storage dtype, converted on the device by the library."""
    if dtype == "f32":
        return proj_f32
    code, tdt = DTYPES[dtype]
    out = torch.empty(proj_f32.shape, dtype=tdt, device=proj_f32.device)
    rct.rct_convert_projections(proj_f32, out, proj_f32.numel(), code, torch.cuda.current_stream())
    return out


def oracle_inputs(proj_f32_host: np.ndarray, dtype: str) -> np.ndarray:
    """The projection values the oracle should see for a storage dtype (oracle rounding)."""
    if dtype == "f16":
        return oracle.round_f16(proj_f32_host)
    if dtype == "bf16":
        return oracle.round_bf16(proj_f32_host)
    return proj_f32_host


def gpu_backproject(w: synth.Workload, proj_dev: torch.Tensor, *, dtype="f32", interp=rct.RCT_INTERP_SOFT,
                    tuning=None, first=0, n=None, chunks=None, frame=rct.RCT_FRAME_GLOBAL,
                    index_rule=rct.RCT_INDEX_FLOOR) -> np.ndarray:
    """Backproject through the C ABI; returns the volume as (L, L, L) float32 numpy."""
    n = w.n_views if n is None else n
    stream = torch.cuda.current_stream()
    with rct.Backprojector(w.L, w.geom.det_w, w.geom.det_h, w.n_views) as bp:
        bp.set_geometry(w.geom.matrices, w.origin, w.spacing)
        bp.set_precision(DTYPES[dtype][0], interp)
        bp.set_frame(frame)
        bp.set_index_rule(index_rule)
        if tuning:
            bp.set_tuning(**tuning)
        data = stored(proj_dev, dtype)
        bounds = chunks or [(first, first + n)]
        for a, b in bounds:
            bp.backproject(data[a - first:b - first], a, b - a, stream)
        out = torch.empty((w.L, w.L, w.L), dtype=torch.float32, device=proj_dev.device)
        bp.read_volume(out, stream)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def oracle_volume(w: synth.Workload, proj_host: np.ndarray, first=0, n=None, threads=None,
                  index_rule=oracle.INDEX_FLOOR) -> np.ndarray:
    n = w.n_views if n is None else n
    threads = threads or oracle.max_threads()
    return oracle.backproject(w.L, w.geom.det_w, w.geom.det_h, w.geom.matrices[first:first + n], w.origin,
                              w.spacing, proj_host, n_threads=threads, index_rule=index_rule)
