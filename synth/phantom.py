"""Analytic ellipsoid phantom, its cone-beam projections and row-wise ramp filtering.

The RabbitCT projections are "filtered and weighted" FP32 images (Section
"RabbitCT Benchmark"); their pre-processing is outside the timed
backprojection.  This module makes a seeded stand-in with the same shape and
character: exact line integrals of random ellipsoids (chord length x density
along each source-to-pixel ray), multiplied by the cosine weight
sdd / |pixel - source|, then convolved along each detector row with the
discrete Shepp-Logan ramp kernel h[n] = -2 / (pi^2 tau^2 (4 n^2 - 1)) (tau =
pixel pitch).  The result has values of both signs and sharp row-wise
gradients at ellipsoid edges.

Computation runs in float64 with torch so that it can use a GPU when one is
present; random parameters come from numpy's seeded PCG64 generator, which is
identical on every platform.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from .geometry import ScanGeometry


@dataclass
class Phantom:
    centers: np.ndarray     # (m, 3) mm
    semi_axes: np.ndarray   # (m, 3) mm
    rotations: np.ndarray   # (m, 3, 3); column k is the direction of semi-axis k
    densities: np.ndarray   # (m,)

    def density_at(self, points: np.ndarray) -> np.ndarray:
        """Phantom value (sum of densities of the ellipsoids containing each point)."""
        p = np.asarray(points, dtype=np.float64)
        out = np.zeros(p.shape[:-1])
        for c, a, q, rho in zip(self.centers, self.semi_axes, self.rotations, self.densities):
            local = ((p - c) @ q) / a
            out += rho * (np.sum(local * local, axis=-1) <= 1.0)
        return out


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_phantom(n_ellipsoids: int = 10, seed: int = 1401, *, radius: float = 100.0,
                   axis_range=(10.0, 60.0), density_range=(0.1, 1.0)) -> Phantom:
    """Seeded ellipsoids: centres uniform in a ball of ``radius`` mm, semi-axes
    uniform in ``axis_range``, uniform random orientation, densities uniform in
    ``density_range``."""
    rng = np.random.default_rng(seed + 7919)
    dirs = rng.normal(size=(n_ellipsoids, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    centers = dirs * (radius * rng.uniform(size=(n_ellipsoids, 1)) ** (1.0 / 3.0))
    axes = rng.uniform(axis_range[0], axis_range[1], size=(n_ellipsoids, 3))
    rots = np.stack([_random_rotation(rng) for _ in range(n_ellipsoids)])
    dens = rng.uniform(density_range[0], density_range[1], size=n_ellipsoids)
    return Phantom(centers, axes, rots, dens)


def project_phantom(geom: ScanGeometry, phantom: Phantom, views, device="cpu") -> torch.Tensor:
    """Line integrals (mm x density) along source-to-pixel rays, float64, shape (len(views), H, W)."""
    dev = torch.device(device)
    f64 = torch.float64
    ii = torch.arange(geom.det_w, device=dev, dtype=f64)
    jj = torch.arange(geom.det_h, device=dev, dtype=f64)
    out = torch.zeros((len(views), geom.det_h, geom.det_w), device=dev, dtype=f64)
    for n, k in enumerate(views):
        u0, v0 = geom.principal[k]
        du = (ii - u0) * geom.pitch                       # (W,)
        dv = (jj - v0) * geom.pitch                       # (H,)
        norm = torch.sqrt(geom.sdd ** 2 + du[None, :] ** 2 + dv[:, None] ** 2)   # (H, W)
        s = geom.source[k]
        for c, a, q, rho in zip(phantom.centers, phantom.semi_axes, phantom.rotations, phantom.densities):
            m = (q / a[None, :]).T                        # world -> unit-sphere frame
            p0 = m @ (s - c)
            alpha = m @ (geom.sdd * geom.d_hat[k])
            beta = m @ (geom.pitch * geom.e_u[k])
            gamma = m @ (geom.pitch * geom.e_v[k])
            # unnormalised direction D(i, j) = alpha + (i-u0) beta + (j-v0) gamma
            dd = [alpha[t] + (ii - u0)[None, :] * beta[t] + (jj - v0)[:, None] * gamma[t] for t in range(3)]
            d2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]
            pd = p0[0] * dd[0] + p0[1] * dd[1] + p0[2] * dd[2]
            cc = float(p0 @ p0) - 1.0
            disc = torch.clamp(pd * pd - d2 * cc, min=0.0)
            out[n] += rho * 2.0 * torch.sqrt(disc) * norm / d2
    return out


def cosine_weight(geom: ScanGeometry, views, device="cpu") -> torch.Tensor:
    """sdd / |pixel - source| per pixel, float64, shape (len(views), H, W)."""
    dev = torch.device(device)
    f64 = torch.float64
    ii = torch.arange(geom.det_w, device=dev, dtype=f64)
    jj = torch.arange(geom.det_h, device=dev, dtype=f64)
    out = torch.empty((len(views), geom.det_h, geom.det_w), device=dev, dtype=f64)
    for n, k in enumerate(views):
        u0, v0 = geom.principal[k]
        du = (ii - u0) * geom.pitch
        dv = (jj - v0) * geom.pitch
        out[n] = geom.sdd / torch.sqrt(geom.sdd ** 2 + du[None, :] ** 2 + dv[:, None] ** 2)
    return out


def shepp_logan_kernel(n_taps: int, pitch: float) -> np.ndarray:
    """Discrete Shepp-Logan ramp kernel h[n], n = -(n_taps-1) .. n_taps-1."""
    n = np.arange(-(n_taps - 1), n_taps, dtype=np.float64)
    return -2.0 / (np.pi ** 2 * pitch ** 2 * (4.0 * n * n - 1.0))


def ramp_filter_rows(proj: torch.Tensor, pitch: float) -> torch.Tensor:
    """Linear (zero-padded) convolution of every row with the Shepp-Logan kernel, scaled by pitch."""
    w = proj.shape[-1]
    npad = 1 << int(np.ceil(np.log2(2 * w - 1)))
    h = np.zeros(npad)
    taps = shepp_logan_kernel(w, pitch)                   # index w-1 is n = 0
    h[:w] = taps[w - 1:]                                  # n = 0 .. w-1
    h[npad - (w - 1):] = taps[:w - 1]                     # n = -(w-1) .. -1
    hf = torch.fft.rfft(torch.from_numpy(h).to(proj.device))
    g = torch.fft.rfft(proj, n=npad, dim=-1)
    return torch.fft.irfft(g * hf, n=npad, dim=-1)[..., :w] * pitch


def make_projections(geom: ScanGeometry, phantom: Phantom, *, device="cpu", views=None,
                     chunk: int = 8, weighted: bool = True, filtered: bool = True,
                     out_device=None) -> torch.Tensor:
    """Pre-processed FP32 projections (n, H, W): line integrals, cosine weight, ramp filter."""
    if views is None:
        views = list(range(geom.n_views))
    out_device = torch.device(device if out_device is None else out_device)
    out = torch.empty((len(views), geom.det_h, geom.det_w), dtype=torch.float32, device=out_device)
    for s in range(0, len(views), chunk):
        vs = views[s:s + chunk]
        p = project_phantom(geom, phantom, vs, device=device)
        if weighted:
            p = p * cosine_weight(geom, vs, device=device)
        if filtered:
            p = ramp_filter_rows(p, geom.pitch)
        out[s:s + len(vs)] = p.to(torch.float32).to(out_device)
    return out
