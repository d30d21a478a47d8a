"""Named workload recipes (volume size, views, detector, seeds).

Full-size recipes follow the RabbitCT shapes: 496 views of 1248x960 FP32
projections and an L^3 FP32 volume with isotropic spacing 256 mm / L centred
on the isocentre.  Reduced recipes shrink the detector but scale the pixel
pitch so that the detector still covers the same field of view (about
240 x 185 mm at the isocentre against a 256 mm cube), so the same fraction of
voxel-view pairs falls partly or fully off the detector.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .geometry import ScanGeometry, short_scan, volume_grid
from .phantom import Phantom, random_phantom, make_projections

FULL_W, FULL_H, FULL_PITCH, FULL_VIEWS = 1248, 960, 0.308, 496


@dataclass
class Workload:
    name: str
    L: int
    geom: ScanGeometry
    origin: np.ndarray
    spacing: np.ndarray
    phantom: Phantom
    seed: int
    extra: dict = field(default_factory=dict)

    @property
    def n_views(self) -> int:
        return self.geom.n_views

    @property
    def updates(self) -> int:
        """Voxel updates of one full backprojection: L^3 x n_views."""
        return self.L ** 3 * self.geom.n_views

    def projections(self, device="cpu", views=None, out_device=None) -> torch.Tensor:
        return make_projections(self.geom, self.phantom, device=device, views=views,
                                out_device=out_device)

    def describe(self) -> dict:
        g = self.geom
        return {"L": self.L, "n_views": g.n_views, "det_w": g.det_w, "det_h": g.det_h,
                "pitch_mm": g.pitch, "sid_mm": g.sid, "sdd_mm": g.sdd, "seed": self.seed,
                "phantom": f"{len(self.phantom.densities)} ellipsoids"}


def make_workload(L: int, n_views: int = FULL_VIEWS, det_w: int = FULL_W, det_h: int = FULL_H,
                  seed: int = 1401, name: str | None = None, n_ellipsoids: int = 10,
                  integer_principal: bool = False) -> Workload:
    pitch = FULL_PITCH * FULL_W / det_w
    geom = short_scan(n_views, det_w, det_h, pitch=pitch, seed=seed,
                      integer_principal=integer_principal)
    origin, spacing = volume_grid(L)
    ph = random_phantom(n_ellipsoids, seed=seed)
    return Workload(name or f"L{L}x{n_views}_{det_w}x{det_h}", L, geom, origin, spacing, ph, seed)


# The configurations measured on the GPU, by name (seed = 1401 + index).
WORKLOADS = {
    "fp32_L128": dict(L=128, seed=1401),
    "fp32_L512": dict(L=512, seed=1402),
    "fp32_L1024": dict(L=1024, seed=1403),
    "prec_L512": dict(L=512, seed=1404),
    # a short scan of the L=512 geometry for profiler captures (inputs still larger than L2)
    "profile_L512": dict(L=512, seed=1402, n_views=64),
    # a few seconds of work anywhere: the benchmark's own plumbing under test, on the CPU
    "tiny_L16": dict(L=16, seed=1410, n_views=8, det_w=64, det_h=48),
}


def named(name: str) -> Workload:
    kw = dict(WORKLOADS[name])
    return make_workload(kw.pop("L"), name=name, **kw)
