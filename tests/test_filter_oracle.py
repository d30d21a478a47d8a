"""Pins for the pre-processing oracle (cosine weight + Shepp-Logan ramp filter), written from the
definitions and from mathematics, not from the oracle's code."""
import numpy as np
import pytest
import scipy.signal

import synth
from oracle import filter as of


def test_delta_row_reproduces_the_kernel():
    """A unit impulse at column m filters to tau * h[i - m], with h[0] = 2 / (pi^2 tau^2) and
    h[+-1] = -2 / (3 pi^2 tau^2)."""
    W, m, tau = 11, 4, 0.5
    row = np.zeros(W)
    row[m] = 1.0
    out = of.ramp_filter_rows(row, tau)
    assert out[m] == pytest.approx(tau * 2.0 / (np.pi ** 2 * tau ** 2), rel=1e-15)
    assert out[m - 1] == pytest.approx(-tau * 2.0 / (3.0 * np.pi ** 2 * tau ** 2), rel=1e-15)
    assert out[m + 1] == pytest.approx(out[m - 1], rel=1e-15)
    assert np.all(out[np.arange(W) != m] < 0.0)            # every off-centre tap is negative


def test_constant_row_closed_form():
    """For a constant row c of length W, the kernel's partial sums telescope
    (sum_{n >= m} 1 / (4 n^2 - 1) = 1 / (2 (2m - 1))) and the whole kernel sums to zero, so
    q(i) = c / (pi^2 tau) * (1 / (2i + 1) + 1 / (2W - 2i - 1))."""
    W, tau, c = 257, 0.308, 3.25
    out = of.ramp_filter_rows(np.full(W, c), tau)
    i = np.arange(W)
    expect = c / (np.pi ** 2 * tau) * (1.0 / (2 * i + 1) + 1.0 / (2 * W - 2 * i - 1))
    np.testing.assert_allclose(out, expect, rtol=1e-11)


def test_brute_force_double_loop():
    rng = np.random.default_rng(5)
    W, tau = 9, 1.7
    rows = rng.normal(size=(3, W))
    expect = np.zeros_like(rows)
    for r in range(3):
        for i in range(W):
            s = 0.0
            for k in range(W):
                d = i - k
                s += rows[r, k] * (-2.0 / (np.pi ** 2 * tau ** 2 * (4.0 * d * d - 1.0)))
            expect[r, i] = tau * s
    np.testing.assert_allclose(of.ramp_filter_rows(rows, tau), expect, rtol=1e-13, atol=1e-15)


def test_matches_fft_convolution():
    """scipy's FFT convolution (a different algorithm) of the zero-padded row with the kernel."""
    rng = np.random.default_rng(6)
    W, tau = 1248, 0.308
    rows = rng.normal(size=(4, W))
    n = np.arange(-(W - 1), W)
    h = -2.0 / (np.pi ** 2 * tau ** 2 * (4.0 * n * n - 1.0))
    expect = np.stack([scipy.signal.fftconvolve(r, h)[W - 1:2 * W - 1] for r in rows]) * tau
    got = of.ramp_filter_rows(rows, tau)
    assert np.max(np.abs(got - expect)) <= 1e-10 * np.max(np.abs(expect))


def test_linearity():
    rng = np.random.default_rng(7)
    a, b = rng.normal(size=(2, 5, 64))
    lhs = of.ramp_filter_rows(2.5 * a - 0.75 * b, 0.4)
    rhs = 2.5 * of.ramp_filter_rows(a, 0.4) - 0.75 * of.ramp_filter_rows(b, 0.4)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_cosine_weight_is_the_ray_angle():
    """D / |pixel - source| equals the cosine between the ray to the pixel and the principal ray,
    computed from the 3D scan geometry (source, principal direction, detector axes)."""
    geom = synth.short_scan(3, 40, 30, pitch=2.0, seed=9)
    for k in range(geom.n_views):
        jj, ii = np.meshgrid(np.arange(geom.det_h), np.arange(geom.det_w), indexing="ij")
        X = geom.pixel_world(k, ii, jj)
        ray = X - geom.source[k]
        cos3d = (ray @ geom.d_hat[k]) / np.linalg.norm(ray, axis=-1)
        u0, v0 = geom.principal[k]
        got = of.cosine_weight(geom.det_w, geom.det_h, geom.sdd, geom.pitch, u0, v0)
        np.testing.assert_allclose(got, cos3d, rtol=1e-12)
        assert got.max() <= 1.0 and got.min() > 0.0


def test_preprocess_is_weight_then_filter():
    rng = np.random.default_rng(8)
    raw = rng.normal(size=(2, 6, 16))
    pp = np.array([[7.5, 2.25], [8.0, 3.0]])
    got = of.preprocess(raw, 1200.0, 0.5, pp)
    for v in range(2):
        w = of.cosine_weight(16, 6, 1200.0, 0.5, *pp[v])
        np.testing.assert_array_equal(got[v], of.ramp_filter_rows(raw[v] * w, 0.5))
