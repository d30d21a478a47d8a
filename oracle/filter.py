"""FP64 oracle for the pre-processing step before the backprojection (test infrastructure only).

TEST INFRASTRUCTURE ONLY: loaded by the test suite and by the benchmark's CPU legs, never by the
product path, and it imports nothing from the product path or from the input generators.

The paper's projections arrive cosine-weighted and ramp-filtered (Section "RabbitCT Benchmark");
this module states that step for raw line integrals p, as the FDK method defines it, with D the
source-detector distance, tau the detector pixel pitch and (u0, v0) the view's principal point:

  cosine weight  p'(i, j) = p(i, j) * D / sqrt(D^2 + ((i - u0) tau)^2 + ((j - v0) tau)^2)
  ramp filter    q(i, j)  = tau * sum_{k=0}^{W-1} h[i - k] p'(k, j)
                 h[n]     = -2 / (pi^2 tau^2 (4 n^2 - 1))        (Shepp-Logan kernel)

The convolution is linear: the row is zero outside [0, W).  It is computed here directly, one row
at a time, with numpy's convolve (a library primitive for the plain sum above).
"""
from __future__ import annotations

import numpy as np


def shepp_logan(n, pitch: float) -> np.ndarray:
    """h[n] for integer n (array-like)."""
    n = np.asarray(n, dtype=np.float64)
    return -2.0 / (np.pi ** 2 * pitch ** 2 * (4.0 * n * n - 1.0))


def cosine_weight(W: int, H: int, sdd: float, pitch: float, u0: float, v0: float) -> np.ndarray:
    """(H, W) array of D / sqrt(D^2 + ((i - u0) tau)^2 + ((j - v0) tau)^2)."""
    du = (np.arange(W, dtype=np.float64) - u0) * pitch
    dv = (np.arange(H, dtype=np.float64) - v0) * pitch
    return sdd / np.sqrt(sdd * sdd + du[None, :] ** 2 + dv[:, None] ** 2)


def ramp_filter_rows(rows, pitch: float) -> np.ndarray:
    """tau * (h * row) restricted to the row's W samples, for every row (last axis), FP64."""
    x = np.asarray(rows, dtype=np.float64)
    W = x.shape[-1]
    h = shepp_logan(np.arange(-(W - 1), W), pitch)        # h[n], n = -(W-1) .. W-1
    flat = x.reshape(-1, W)
    out = np.empty_like(flat)
    for r in range(flat.shape[0]):
        # full convolution index m = i + (W - 1) pairs row[k] with h[i - k]
        out[r] = np.convolve(flat[r], h)[W - 1:2 * W - 1]
    return (out * pitch).reshape(x.shape)


def preprocess(raw, sdd: float, pitch: float, principal) -> np.ndarray:
    """Cosine weight then ramp filter of raw projections (n, H, W); principal is (n, 2) (u0, v0)."""
    raw = np.asarray(raw, dtype=np.float64)
    n, H, W = raw.shape
    pp = np.asarray(principal, dtype=np.float64).reshape(n, 2)
    out = np.empty_like(raw)
    for v in range(n):
        out[v] = ramp_filter_rows(raw[v] * cosine_weight(W, H, sdd, pitch, pp[v, 0], pp[v, 1]), pitch)
    return out
