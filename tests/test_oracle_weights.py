"""Pins of the oracle's weight functions against closed forms (Sec. 3, Sec. 5.1)."""
import numpy as np
import pytest

import oracle

THETA = 3 * np.pi / 8


@pytest.mark.parametrize("alpha,expected", [
    (0.0, 1.0),                    # exclusive zone
    (np.pi / 2 - THETA, 1.0),      # edge of the exclusive zone
    (np.pi / 4, 0.5),              # middle of the blend zone of two neighbouring axes
    (THETA, 0.0),                  # angular threshold (Eq. angular_threshold)
    (np.pi / 2, 0.0),              # orthogonal
    (np.pi, 0.0),                  # opposite
])
def test_w_dir_closed_form(alpha, expected):
    assert oracle.w_dir(np.cos(alpha), THETA) == pytest.approx(expected, abs=1e-12)


def test_w_dir_linear_in_angle_over_full_range():
    # the blend zone maps linearly onto [0, 1] (Sec. 3 text after Eq. direction_weight)
    a = np.linspace(np.pi / 2 - THETA, THETA, 17)
    w = np.array([oracle.w_dir(np.cos(x), THETA) for x in a])
    assert w[0] == pytest.approx(1.0) and w[-1] == pytest.approx(0.0, abs=1e-12)
    assert np.allclose(np.diff(w), np.diff(w)[0], atol=1e-12)


@pytest.mark.parametrize("theta", [THETA, 0.3 * np.pi, 0.45 * np.pi])
def test_w_dir_partition_of_unity_in_coordinate_plane(theta):
    # a normal in the X/Y plane splits its weight between X+ and Y+ with sum 1
    for alpha in np.linspace(0, np.pi / 2, 41):
        n = np.array([np.cos(alpha), np.sin(alpha), 0.0])
        s = oracle.w_dir(n[0], theta) + oracle.w_dir(n[1], theta)
        assert s == pytest.approx(1.0, abs=1e-12)


def test_every_normal_matches_a_direction_at_default_theta():
    # Eq. angular_threshold: with theta > acos(1/sqrt 3) every normal belongs to >= 1 direction
    rng = np.random.default_rng(0)
    n = rng.normal(size=(5000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    for v in n:
        cnt = sum(oracle.w_dir(s * v[a], THETA) > 0 for a in range(3) for s in (1, -1))
        assert 1 <= cnt <= 3


def test_w_icp_range():
    # Eq. ICP_weight stays in [0, 1] for z >= z_min and equals 1 at z_min
    zmin = 0.1
    z = np.linspace(zmin, 6.0, 100)
    w = 1.0 / (z + (1.0 - zmin)) ** 2
    assert w[0] == pytest.approx(1.0) and np.all((w > 0) & (w <= 1))
