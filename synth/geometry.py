"""C-arm short-scan geometry: one 3x4 projection matrix per view.

The RabbitCT dataset gives every projection image its own matrix
A_i in R^{3x4} (Section "RabbitCT Benchmark").  A world point X (mm) maps to
homogeneous detector coordinates (u, v, w) = A_i (X, 1); the pixel hit is
(u/w, v/w) and w approximates the source-to-voxel distance (Section
"Algorithm").  Here the matrices are synthesised from an explicit pinhole
model so that tests can recompute the same mapping without the matrix:

  * circular short scan over ``arc_deg`` degrees, view angles spaced evenly
    from -arc/2 to +arc/2;
  * source at distance ``sid`` from the isocentre (the world origin),
    detector at distance ``sdd`` from the source, square pixels of ``pitch``;
  * every view gets a small rigid tilt of the whole source-detector pair
    about a random axis through the isocentre (|angle| <= ``tilt_deg``), so
    the principal ray still passes through the isocentre;
  * principal point = detector centre ((W-1)/2, (H-1)/2) plus a uniform
    jitter of up to ``jitter_px`` pixels per axis.

Pixel (i, j) is the sample at detector coordinate (i, j): column i along
e_u, row j along e_v, row-major storage with row stride W.  The third matrix
row is (d^T, -d.s) with d the unit principal direction and s the source, so
w is the depth along the principal axis in mm.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class ScanGeometry:
    n_views: int
    det_w: int
    det_h: int
    pitch: float            # mm per pixel
    sid: float              # source - isocentre distance, mm
    sdd: float              # source - detector distance, mm
    angles: np.ndarray      # (n,) rad
    source: np.ndarray      # (n, 3) mm
    e_u: np.ndarray         # (n, 3) unit detector column direction
    e_v: np.ndarray         # (n, 3) unit detector row direction
    d_hat: np.ndarray       # (n, 3) unit principal direction (source -> isocentre)
    principal: np.ndarray   # (n, 2) principal point (u0, v0) in pixels
    matrices: np.ndarray    # (n, 3, 4) float64 row-major projection matrices
    seed: int

    @property
    def focal_px(self) -> float:
        return self.sdd / self.pitch

    def pixel_world(self, view: int, i, j):
        """World position (mm) of detector sample (i, j) of ``view``."""
        i = np.asarray(i, dtype=np.float64)
        j = np.asarray(j, dtype=np.float64)
        u0, v0 = self.principal[view]
        c = self.source[view] + self.sdd * self.d_hat[view]
        return (c + ((i - u0) * self.pitch)[..., None] * self.e_u[view]
                + ((j - v0) * self.pitch)[..., None] * self.e_v[view])


def _rotation(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rodrigues rotation matrix about unit ``axis`` by ``angle`` rad."""
    a = axis / np.linalg.norm(axis)
    k = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + np.sin(angle) * k + (1.0 - np.cos(angle)) * (k @ k)


def short_scan(n_views: int = 496, det_w: int = 1248, det_h: int = 960, *,
               sid: float = 750.0, sdd: float = 1200.0, pitch: float = 0.308,
               arc_deg: float = 200.0, tilt_deg: float = 0.5, jitter_px: float = 2.0,
               seed: int = 1401, integer_principal: bool = False) -> ScanGeometry:
    """Build the seeded short-scan geometry described in the module docstring.

    ``integer_principal`` rounds the jittered principal point to whole pixels
    (used by tests that put a single bright pixel exactly on it).
    """
    if n_views <= 0 or det_w <= 0 or det_h <= 0:
        raise ValueError("n_views, det_w and det_h must be positive")
    rng = np.random.default_rng(seed)
    if n_views == 1:
        angles = np.zeros(1)
    else:
        angles = np.deg2rad(-arc_deg / 2.0 + np.arange(n_views) * (arc_deg / (n_views - 1)))
    tilt_axes = rng.normal(size=(n_views, 3))
    tilt_angles = np.deg2rad(rng.uniform(-tilt_deg, tilt_deg, size=n_views))
    jitter = rng.uniform(-jitter_px, jitter_px, size=(n_views, 2))

    source = np.empty((n_views, 3))
    e_u = np.empty((n_views, 3))
    e_v = np.empty((n_views, 3))
    d_hat = np.empty((n_views, 3))
    principal = np.empty((n_views, 2))
    mats = np.empty((n_views, 3, 4))
    f = sdd / pitch
    for k in range(n_views):
        th = angles[k]
        s = sid * np.array([np.cos(th), np.sin(th), 0.0])
        eu = np.array([-np.sin(th), np.cos(th), 0.0])
        ev = np.array([0.0, 0.0, 1.0])
        rt = _rotation(tilt_axes[k], tilt_angles[k])
        s, eu, ev = rt @ s, rt @ eu, rt @ ev
        d = -s / np.linalg.norm(s)
        u0 = (det_w - 1) / 2.0 + jitter[k, 0]
        v0 = (det_h - 1) / 2.0 + jitter[k, 1]
        if integer_principal:
            u0, v0 = float(np.round(u0)), float(np.round(v0))
        r = np.stack([eu, ev, d])                     # world -> camera rotation
        kmat = np.array([[f, 0.0, u0], [0.0, f, v0], [0.0, 0.0, 1.0]])
        mats[k] = kmat @ np.concatenate([r, (-r @ s)[:, None]], axis=1)
        source[k], e_u[k], e_v[k], d_hat[k] = s, eu, ev, d
        principal[k] = (u0, v0)
    return ScanGeometry(n_views, det_w, det_h, pitch, sid, sdd, angles, source, e_u, e_v,
                        d_hat, principal, mats, seed)


def volume_grid(L: int, fov_mm: float = 256.0):
    """Centred isotropic voxel grid: returns (origin[3], spacing[3]) in mm.

    ``origin`` is the world position of the centre of voxel (0, 0, 0); voxel
    centres are symmetric about the isocentre, spacing = fov / L.
    """
    if L <= 0:
        raise ValueError("L must be positive")
    sp = fov_mm / L
    origin = np.full(3, -(L - 1) / 2.0 * sp)
    return origin, np.full(3, sp)


def orthographic_matrix(origin, spacing, shift=(0.0, 0.0)) -> np.ndarray:
    """A 3x4 matrix with w == 1 that maps voxel (x, y, z) to pixel (x + du, y + dv).

    Used by closed-form tests: with it a single view backprojects the image
    itself (shifted by ``shift``) into every z-plane.
    """
    o = np.asarray(origin, dtype=np.float64)
    s = np.asarray(spacing, dtype=np.float64)
    du, dv = shift
    return np.array([[1.0 / s[0], 0.0, 0.0, -o[0] / s[0] + du],
                     [0.0, 1.0 / s[1], 0.0, -o[1] / s[1] + dv],
                     [0.0, 0.0, 0.0, 1.0]])
