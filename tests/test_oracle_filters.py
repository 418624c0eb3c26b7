"""Pins of the oracle's bilateral input filters, Sec. 7 normals and post-fusion error
(oracle/filters.py) against closed forms, invariants and scipy's correlation."""
import numpy as np
import pytest
import scipy.ndimage

from oracle import filters as F
import scenes

K = scenes.Intrinsics(64, 48, 60.0, 60.0, 31.5, 23.5)


def _gauss(r, sd):
    d = np.arange(-r, r + 1)
    return np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * sd * sd))


def test_depth_filter_keeps_constant_depth_and_holes():
    rng = np.random.default_rng(0)
    z = np.full((48, 64), 1.7)
    z[rng.random(z.shape) < 0.2] = 0.0
    out = F.bilateral_depth(z, 5, 5.0, 0.025)
    assert np.array_equal(out == 0, z == 0)
    np.testing.assert_allclose(out[z > 0], 1.7, rtol=1e-14)


def test_depth_filter_keeps_a_linear_ramp_inside():
    """Window weights are symmetric for a linear ramp, so the weighted mean is the centre value."""
    v, u = np.mgrid[0:48, 0:64]
    z = 1.0 + 0.001 * u + 0.0005 * v
    out = F.bilateral_depth(z, 5, 5.0, 0.025)
    np.testing.assert_allclose(out[5:-5, 5:-5], z[5:-5, 5:-5], rtol=0, atol=1e-13)
    assert np.max(np.abs(out - z)) > 1e-4  # the border, where the window is one-sided, moves


def test_depth_filter_does_not_cross_a_step():
    z = np.full((48, 64), 1.0)
    z[:, 32:] = 1.2  # 8 sigma_r
    out = F.bilateral_depth(z, 5, 5.0, 0.025)
    np.testing.assert_allclose(out[:, :32], 1.0, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out[:, 32:], 1.2, rtol=0, atol=1e-13)


def test_depth_filter_without_range_term_is_a_normalised_gaussian():
    rng = np.random.default_rng(1)
    z = 1.0 + 0.05 * rng.random((48, 64))
    out = F.bilateral_depth(z, 4, 2.0, 1e9)
    G = _gauss(4, 2.0)
    ref = scipy.ndimage.correlate(z, G, mode="constant") / scipy.ndimage.correlate(np.ones_like(z), G, mode="constant")
    np.testing.assert_allclose(out, ref, rtol=1e-12)


def _plane_points(n, d):
    """Points of the plane <n, x> = d seen by K (exact)."""
    v, u = np.mgrid[0:K.height, 0:K.width]
    ray = np.stack([(u - K.cx) / K.fx, (v - K.cy) / K.fy, np.ones(u.shape)], -1)
    t = d / (ray @ n)
    return ray * t[..., None], t


def test_normals_of_a_plane_are_its_normal():
    n = np.array([0.3, -0.2, -1.0])
    n /= np.linalg.norm(n)
    P, z = _plane_points(n, -1.5)
    nn, has = F.normals(P, z > 0)
    assert has[1:-1, 1:-1].all() and not has[0].any() and not has[:, -1].any()
    np.testing.assert_allclose(nn[has], np.broadcast_to(n, nn[has].shape), atol=1e-12)


def test_normal_filter_keeps_planes_and_a_right_angle_crease():
    n1 = np.array([0.0, 0.0, -1.0])
    n2 = np.array([-1.0, 0.0, 0.0])
    nn = np.zeros((48, 64, 3))
    nn[:, :30] = n1
    nn[:, 30:] = n2
    has = np.ones((48, 64), bool)
    has[:, 10] = False
    out = F.bilateral_normals(nn, has, 5, 2.5, 5.0)
    w90 = np.exp(-(90.0 ** 2) / (2 * 5.0 ** 2))
    assert np.max(np.abs(out[has] - nn[has])) < 10 * w90 + 1e-15
    assert not out[~has].any()


def test_normal_filter_without_range_term_is_a_normalised_gaussian():
    rng = np.random.default_rng(2)
    nn = np.array([0.0, 0.0, -1.0]) + 0.2 * rng.standard_normal((48, 64, 3))
    nn /= np.linalg.norm(nn, axis=-1, keepdims=True)
    has = np.ones((48, 64), bool)
    out = F.bilateral_normals(nn, has, 3, 1.5, 1e9)
    G = _gauss(3, 1.5)
    ref = np.stack([scipy.ndimage.correlate(nn[..., a], G, mode="constant") for a in range(3)], -1)
    ref /= np.linalg.norm(ref, axis=-1, keepdims=True)
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_depth_mae_closed_form():
    rng = np.random.default_rng(3)
    a = 1.0 + rng.random((48, 64))
    b = a + 0.003
    a[rng.random(a.shape) < 0.1] = 0
    b[rng.random(b.shape) < 0.1] = 0
    s, c = F.depth_mae(a, b)
    both = (a > 0) & (b > 0)
    assert c == int(both.sum())
    assert s / c == pytest.approx(0.003, rel=1e-9)
