"""Pins for the FP64 oracle, written independently of its code.

Each check takes a loaded oracle library (ctypes) and raises AssertionError
when the oracle disagrees with a fact fixed by the paper's definition of the
backprojection (Section "Algorithm", Listing 1) or by mathematics:

* orthographic special cases (w == 1, pixel = voxel + shift) where one view
  backprojects the image itself, or its bilinear resampling, which
  ``scipy.ndimage.map_coordinates(order=1, mode="grid-constant")`` computes
  as a library routine on the zero-extended grid;
* cone-beam geometry recomputed from the pinhole model (source, detector
  axes, principal point) instead of the 3x4 matrix, interpolated by scipy;
* a brute-force sum of separable tent weights over every pixel;
* exact reproduction of an affine image, the constant-image law c * 1/w^2
  inside the detector and 0 outside, the isocentre landing on the principal
  point with weight 1/sid^2, linearity, and additivity over view splits.

The mutation test in ``test_oracle_mutations.py`` plants plausible mistakes
in copies of the oracle and checks that these pins catch each one.
"""
from __future__ import annotations

import numpy as np
import scipy.ndimage as ndi

import oracle
import synth

# Reduced detector, full-size field of view (see synth.workloads).
SMALL_W, SMALL_H = 24, 18


def _small_geom(n_views=5, seed=11, integer_principal=False, W=SMALL_W, H=SMALL_H):
    pitch = synth.workloads.FULL_PITCH * synth.workloads.FULL_W / W
    return synth.short_scan(n_views, W, H, pitch=pitch, seed=seed, integer_principal=integer_principal)


def voxel_world(L, origin, spacing):
    """World coordinates (L, L, L, 3) of voxel centres, indexed [z, y, x]."""
    ax = [origin[k] + np.arange(L) * spacing[k] for k in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([x, y, z], axis=-1)


def pinhole(geom, k, X):
    """Detector coordinates (ix, iy) and depth w of world points X for view k, from the
    source/detector description (ray-plane intersection), not from the matrix."""
    s, d = geom.source[k], geom.d_hat[k]
    rel = X - s
    depth = rel @ d
    hit = s + (geom.sdd / depth)[..., None] * rel
    c = s + geom.sdd * d
    ix = geom.principal[k, 0] + (hit - c) @ geom.e_u[k] / geom.pitch
    iy = geom.principal[k, 1] + (hit - c) @ geom.e_v[k] / geom.pitch
    return ix, iy, depth


def bilinear_scipy(img, ix, iy):
    """Bilinear value on the zero-extended pixel grid (library routine)."""
    coords = np.stack([np.ravel(iy), np.ravel(ix)])
    out = ndi.map_coordinates(np.asarray(img, np.float64), coords, order=1,
                              mode="grid-constant", cval=0.0, prefilter=False)
    return out.reshape(np.shape(ix))


def bilinear_tent(img, ix, iy):
    """Brute force: sum over all pixels of I[j, i] * tent(ix - i) * tent(iy - j)."""
    H, W = img.shape
    hx = np.maximum(0.0, 1.0 - np.abs(np.ravel(ix)[:, None] - np.arange(W)[None, :]))
    hy = np.maximum(0.0, 1.0 - np.abs(np.ravel(iy)[:, None] - np.arange(H)[None, :]))
    return np.einsum("vj,ji,vi->v", hy, np.asarray(img, np.float64), hx).reshape(np.shape(ix))


def _run(lib, L, W, H, mats, origin, spacing, proj):
    return oracle.backproject(L, W, H, mats, origin, spacing, proj, lib=lib)


def _close(a, b, rel, what):
    scale = max(np.max(np.abs(b)), 1e-300)
    err = np.max(np.abs(a - b)) / scale
    assert err <= rel, f"{what}: max error {err:.3e} x max|ref| exceeds {rel:.1e}"


# --------------------------------------------------------------------------- checks

def check_orthographic_identity(lib):
    """w == 1 and pixel == voxel: one view writes I[y][x] into every plane, 0 off the image."""
    rng = np.random.default_rng(1)
    W, H, L = 7, 5, 9
    img = (rng.integers(-64, 64, size=(H, W)) / 8.0).astype(np.float32)
    origin, spacing = np.zeros(3), np.ones(3)
    mat = synth.orthographic_matrix(origin, spacing)
    f = _run(lib, L, W, H, mat[None], origin, spacing, img[None])
    expect = np.zeros((L, L))
    expect[:H, :W] = img
    for z in range(L):
        assert np.array_equal(f[z], expect), "orthographic identity: plane differs from the image"


def check_orthographic_shift(lib):
    """Fractional shifts, including negative ones, equal scipy's zero-extended bilinear."""
    rng = np.random.default_rng(2)
    W, H, L = 7, 5, 9
    img = rng.normal(size=(H, W)).astype(np.float32)
    for origin, spacing, shift in [((0, 0, 0), (1, 1, 1), (-0.375, 1.625)),
                                   ((-3.2, 1.1, 0.4), (0.7, 0.7, 0.7), (0.8125, -0.6875)),
                                   ((0, 0, 0), (1, 1, 1), (-1.25, 3.5))]:
        mat = synth.orthographic_matrix(origin, spacing, shift)
        f = _run(lib, L, W, H, mat[None], origin, spacing, img[None])
        yy, xx = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
        expect = bilinear_scipy(img, xx + shift[0], yy + shift[1])
        for z in range(L):
            _close(f[z], expect, 1e-12, f"orthographic shift {shift}")


def _cone_case(seed, L=7, n_views=5, W=SMALL_W, H=SMALL_H):
    geom = _small_geom(n_views, seed=seed, W=W, H=H)
    origin, spacing = synth.volume_grid(L)
    rng = np.random.default_rng(seed)
    proj = rng.normal(size=(n_views, H, W)).astype(np.float32)
    return geom, origin, spacing, proj


def check_cone_beam_scipy(lib):
    """Short-scan cone beam: pinhole geometry + scipy bilinear + 1/w^2, summed over views."""
    geom, origin, spacing, proj = _cone_case(seed=3)
    L = 7
    f = _run(lib, L, geom.det_w, geom.det_h, geom.matrices, origin, spacing, proj)
    X = voxel_world(L, origin, spacing)
    expect = np.zeros((L, L, L))
    for k in range(geom.n_views):
        ix, iy, w = pinhole(geom, k, X)
        expect += bilinear_scipy(proj[k], ix, iy) / (w * w)
    _close(f, expect, 1e-10, "cone beam vs pinhole + scipy")


def check_tent_brute_force(lib):
    """Same with a rectangular detector (W != H) and a tent-weight sum over every pixel."""
    geom, origin, spacing, proj = _cone_case(seed=4, L=6, n_views=4, W=20, H=29)
    L = 6
    f = _run(lib, L, geom.det_w, geom.det_h, geom.matrices, origin, spacing, proj)
    X = voxel_world(L, origin, spacing)
    expect = np.zeros((L, L, L))
    for k in range(geom.n_views):
        ix, iy, w = pinhole(geom, k, X)
        expect += bilinear_tent(proj[k], ix, iy) / (w * w)
    _close(f, expect, 1e-10, "cone beam vs tent brute force")


def check_affine_image(lib):
    """I(i, j) = a + b i + c j is reproduced exactly wherever all four taps are on the image."""
    geom = _small_geom(6, seed=5)
    L = 9
    origin, spacing = synth.volume_grid(L)
    W, H = geom.det_w, geom.det_h
    a, b, c = 0.5, 0.25, -0.125
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    img = (a + b * ii + c * jj).astype(np.float32)
    X = voxel_world(L, origin, spacing)
    n_inside = 0
    for k in range(geom.n_views):
        f = _run(lib, L, W, H, geom.matrices[k:k + 1], origin, spacing, img[None])
        ix, iy, w = pinhole(geom, k, X)
        eps = 1e-6
        inside = (ix > eps) & (ix < W - 1 - eps) & (iy > eps) & (iy < H - 1 - eps)
        n_inside += int(inside.sum())
        expect = (a + b * ix + c * iy) / (w * w)
        _close(f[inside], expect[inside], 1e-12, "affine image")
    assert n_inside > 100, "affine check saw too few voxels inside the detector"


def check_constant_image(lib):
    """I == c gives c / w^2 inside the detector, 0 where all taps miss, and between in the band."""
    geom = _small_geom(6, seed=6)
    L = 9
    origin, spacing = synth.volume_grid(L)
    W, H = geom.det_w, geom.det_h
    cval = 1.5
    img = np.full((1, H, W), cval, np.float32)
    X = voxel_world(L, origin, spacing)
    n_in = n_out = 0
    for k in range(geom.n_views):
        f = _run(lib, L, W, H, geom.matrices[k:k + 1], origin, spacing, img)
        ix, iy, w = pinhole(geom, k, X)
        eps = 1e-6
        inside = (ix > eps) & (ix < W - 1 - eps) & (iy > eps) & (iy < H - 1 - eps)
        outside = (ix < -1 - eps) | (ix > W + eps) | (iy < -1 - eps) | (iy > H + eps)
        band = ~inside & ~outside
        n_in += int(inside.sum())
        n_out += int(outside.sum())
        _close(f[inside], cval / (w[inside] ** 2), 1e-12, "constant image inside")
        assert np.all(f[outside] == 0.0), "constant image: nonzero where all taps miss"
        assert np.all(f[band] >= 0.0) and np.all(f[band] <= cval / w[band] ** 2 * (1 + 1e-12)), \
            "constant image: band value outside [0, c/w^2]"
    assert n_in > 100 and n_out > 10, "constant-image check needs voxels both on and off the detector"


def check_isocentre_delta(lib):
    """A voxel at the isocentre lands on each view's principal point with w = sid."""
    geom = _small_geom(6, seed=7, integer_principal=True)
    L = 9                                    # odd: the centre voxel sits on the isocentre
    origin, spacing = synth.volume_grid(L)
    W, H = geom.det_w, geom.det_h
    proj = np.zeros((geom.n_views, H, W), np.float32)
    for k in range(geom.n_views):
        u0, v0 = geom.principal[k]
        proj[k, int(v0), int(u0)] = 1.0
    f = _run(lib, L, W, H, geom.matrices, origin, spacing, proj)
    c = L // 2
    expect = geom.n_views / geom.sid ** 2
    assert abs(f[c, c, c] - expect) <= 1e-9 * expect, "isocentre voxel != n_views / sid^2"


def check_linearity(lib):
    """f(2 I1 - 0.5 I2) == 2 f(I1) - 0.5 f(I2) (inputs chosen so the FP32 combination is exact)."""
    geom, origin, spacing, _ = _cone_case(seed=8)
    rng = np.random.default_rng(8)
    shape = (geom.n_views, geom.det_h, geom.det_w)
    i1 = rng.integers(-100, 100, size=shape).astype(np.float32)
    i2 = rng.integers(-100, 100, size=shape).astype(np.float32)
    L = 7
    run = lambda p: _run(lib, L, geom.det_w, geom.det_h, geom.matrices, origin, spacing, p)
    lhs = run((2.0 * i1 - 0.5 * i2).astype(np.float32))
    _close(lhs, 2.0 * run(i1) - 0.5 * run(i2), 1e-12, "linearity")


def check_view_additivity(lib):
    """Backprojecting views [0, k) then [k, n) into the same volume equals one pass over [0, n)."""
    geom, origin, spacing, proj = _cone_case(seed=9)
    L, W, H = 7, geom.det_w, geom.det_h
    whole = _run(lib, L, W, H, geom.matrices, origin, spacing, proj)
    part = oracle.backproject(L, W, H, geom.matrices[:2], origin, spacing, proj[:2], lib=lib)
    oracle.backproject(L, W, H, geom.matrices[2:], origin, spacing, proj[2:], vol=part, lib=lib)
    assert np.array_equal(whole, part), "view split changed the result"
    _close(whole, sum(_run(lib, L, W, H, geom.matrices[k:k + 1], origin, spacing, proj[k:k + 1])
                      for k in range(geom.n_views)), 1e-12, "sum of single-view passes")


def check_voxel_subset(lib):
    """The voxel-list entry point gives the same sums as the volume entry point."""
    geom, origin, spacing, proj = _cone_case(seed=10)
    L, W, H = 7, geom.det_w, geom.det_h
    vol = _run(lib, L, W, H, geom.matrices, origin, spacing, proj)
    idx = np.random.default_rng(10).choice(L ** 3, size=60, replace=False)
    sub = oracle.backproject_voxels(L, W, H, geom.matrices, origin, spacing, proj, idx, lib=lib)
    assert np.array_equal(sub, vol.reshape(-1)[idx]), "voxel subset differs from volume"


def check_zslab(lib):
    """A z-slab [z0, z1) equals the same planes of the full volume (planes are independent)."""
    geom, origin, spacing, proj = _cone_case(seed=12)
    L, W, H = 7, geom.det_w, geom.det_h
    vol = _run(lib, L, W, H, geom.matrices, origin, spacing, proj)
    slab = oracle.backproject(L, W, H, geom.matrices, origin, spacing, proj, z_range=(2, 5),
                              n_threads=2, lib=lib)
    assert np.array_equal(slab, vol[2:5]), "z-slab differs from the full volume"


def check_trunc_orthographic(lib):
    """Listing 1's truncating cell: with w == 1 and pixel = voxel + (-1.25, 2), column x = 1 sits at
    ix = -0.25, truncated to cell 0 with fx = -0.25, so a constant image extrapolates to itself; column
    x = 0 sits at ix = -1.25, cell -1, so only tap 0 contributes, with weight ix + 1 = -0.25.  Floor
    gives 0.75 c and 0 there."""
    W, H, L = 6, 5, 8
    cval = 2.0
    img = np.full((1, H, W), cval, np.float32)
    origin, spacing = np.zeros(3), np.ones(3)
    mat = synth.orthographic_matrix(origin, spacing, (-1.25, 2.0))[None]
    ft = oracle.backproject(L, W, H, mat, origin, spacing, img, lib=lib, index_rule=oracle.INDEX_TRUNC)
    ff = oracle.backproject(L, W, H, mat, origin, spacing, img, lib=lib)
    rows = slice(0, H - 3)                      # iy = y + 2 keeps both tap rows on the image
    assert np.all(ft[:, rows, 1] == cval), "truncated cell at ix = -0.25 must extrapolate the constant"
    assert np.all(ft[:, rows, 0] == -0.25 * cval), "truncated cell at ix = -1.25 must weight tap 0 by -0.25"
    assert np.all(ff[:, rows, 1] == 0.75 * cval) and np.all(ff[:, rows, 0] == 0.0), "floor reference changed"


def check_trunc_affine_extrapolation(lib):
    """Truncation keeps the cell on the image for ix in (-1, 0) (and iy), where the lerp of an affine
    image I = a + b i + c j extrapolates it exactly; elsewhere inside it agrees with floor."""
    geom = _small_geom(6, seed=5)
    L = 9
    origin, spacing = synth.volume_grid(L)
    W, H = geom.det_w, geom.det_h
    a, b, c = 0.5, 0.25, -0.125
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    img = (a + b * ii + c * jj).astype(np.float32)
    X = voxel_world(L, origin, spacing)
    n_band = 0
    for k in range(geom.n_views):
        ft = oracle.backproject(L, W, H, geom.matrices[k:k + 1], origin, spacing, img[None], lib=lib,
                                index_rule=oracle.INDEX_TRUNC)
        ff = _run(lib, L, W, H, geom.matrices[k:k + 1], origin, spacing, img[None])
        ix, iy, w = pinhole(geom, k, X)
        eps = 1e-6
        cover = (ix > -1 + eps) & (ix < W - 1 - eps) & (iy > -1 + eps) & (iy < H - 1 - eps)
        band = cover & ((ix < -eps) | (iy < -eps))
        n_band += int(band.sum())
        _close(ft[cover], ((a + b * ix + c * iy) / (w * w))[cover], 1e-12, "truncated cell, affine image")
        nonneg = (ix > eps) & (iy > eps)
        assert np.array_equal(ft[nonneg], ff[nonneg]), "truncation and floor differ at non-negative coordinates"
    assert n_band > 10, "truncation check saw too few voxels in the negative band"


ALL_CHECKS = [check_orthographic_identity, check_orthographic_shift, check_cone_beam_scipy,
              check_tent_brute_force, check_affine_image, check_constant_image,
              check_isocentre_delta, check_linearity, check_view_additivity,
              check_voxel_subset, check_zslab, check_trunc_orthographic, check_trunc_affine_extrapolation]
