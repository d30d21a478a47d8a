"""The seeded input generator: determinism and closed forms of its geometry and phantom (CPU)."""
import numpy as np
import torch

import synth
from synth.phantom import Phantom, project_phantom


def test_geometry_is_seeded_and_deterministic():
    a = synth.short_scan(8, 64, 48, seed=5)
    b = synth.short_scan(8, 64, 48, seed=5)
    c = synth.short_scan(8, 64, 48, seed=6)
    assert np.array_equal(a.matrices, b.matrices)
    assert not np.array_equal(a.matrices, c.matrices)


def test_isocentre_projects_to_principal_point_at_depth_sid():
    g = synth.short_scan(16, 1248, 960, seed=1401)
    for k in range(g.n_views):
        u, v, w = g.matrices[k] @ np.array([0.0, 0.0, 0.0, 1.0])
        assert abs(u / w - g.principal[k, 0]) < 1e-9 and abs(v / w - g.principal[k, 1]) < 1e-9
        assert abs(w - g.sid) < 1e-9
        assert np.all(np.abs(g.principal[k] - [(1248 - 1) / 2, (960 - 1) / 2]) <= 2.0)


def test_matrix_maps_detector_pixels_to_themselves():
    g = synth.short_scan(4, 40, 30, seed=3)
    for k in range(g.n_views):
        for i, j in [(0, 0), (39, 29), (12.5, 7.25)]:
            X = g.pixel_world(k, i, j)
            u, v, w = g.matrices[k] @ np.append(X, 1.0)
            assert abs(u / w - i) < 1e-9 and abs(v / w - j) < 1e-9 and abs(w - g.sdd) < 1e-9


def test_short_scan_covers_200_degrees_with_bounded_tilt():
    g = synth.short_scan(496, 1248, 960, seed=1402)
    assert np.isclose(np.rad2deg(g.angles[-1] - g.angles[0]), 200.0)
    # the tilt keeps the source on the sphere of radius sid and the principal ray through the isocentre
    assert np.allclose(np.linalg.norm(g.source, axis=1), g.sid)
    assert np.allclose(g.d_hat, -g.source / g.sid)
    # the rotation axis of the scan is tilted by at most 0.5 degrees
    tilt = np.rad2deg(np.arccos(np.clip(g.e_v[:, 2], -1, 1)))
    assert tilt.max() <= 0.5 + 1e-9


def test_volume_grid_is_centred():
    for L in (7, 8, 512):
        o, s = synth.volume_grid(L)
        assert np.allclose(s, 256.0 / L)
        assert np.allclose(o + (L - 1) * s, -o)


def test_sphere_line_integral_closed_form():
    """Through a sphere of radius r the chord at distance d from the centre is 2 sqrt(r^2 - d^2)."""
    g = synth.short_scan(1, 65, 65, pitch=1.0, sdd=1200.0, sid=750.0, tilt_deg=0.0, jitter_px=0.0, seed=0)
    r, rho = 40.0, 0.7
    ph = Phantom(np.zeros((1, 3)), np.full((1, 3), r), np.eye(3)[None], np.array([rho]))
    p = project_phantom(g, ph, [0]).numpy()[0]
    jj, ii = np.meshgrid(np.arange(65), np.arange(65), indexing="ij")
    X = g.pixel_world(0, ii, jj)
    s = g.source[0]
    dirs = (X - s) / np.linalg.norm(X - s, axis=-1, keepdims=True)
    # distance from the isocentre (sphere centre) to each ray
    t = -(s @ dirs.reshape(-1, 3).T).reshape(65, 65)
    closest = s + t[..., None] * dirs
    d = np.linalg.norm(closest, axis=-1)
    expect = rho * 2.0 * np.sqrt(np.clip(r * r - d * d, 0.0, None))
    assert np.allclose(p, expect, atol=1e-9)
    assert p[32, 32] > 0.99 * 2 * r * rho


def test_projections_shape_dtype_and_signs():
    w = synth.make_workload(16, n_views=4, det_w=96, det_h=74, seed=9)
    p = w.projections()
    assert p.shape == (4, 74, 96) and p.dtype == torch.float32
    assert torch.isfinite(p).all()
    assert (p > 0).any() and (p < 0).any()          # the ramp filter makes both signs
    assert torch.equal(p, w.projections())          # deterministic
