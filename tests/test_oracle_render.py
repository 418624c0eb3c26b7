"""Pins of the oracle's ray-cast render (Sec. 4) on analytic scenes."""
import numpy as np
import pytest

import oracle
import scenes


def test_plane_render_is_exact():
    """A fused plane is a linear field; trilinear interpolation and the convex
    combination of directions reproduce it exactly, so the render equals the
    analytic ray-plane intersection up to the float32 depth input."""
    s = scenes.plane_scene()
    P = oracle.Params(voxel_size=0.01, truncation=0.04)
    m = oracle.OracleMap(P)
    for i in range(4):
        f = s.frame(i)
        m.integrate(f.depth, f.rgb, s.K, f.pose)
    T = s.poses[1].copy()
    T[:3, 3] += np.array([0.01, -0.02, 0.01])
    d, n, c, cok = m.render(s.K, T)
    ex = s.render(T, noise=False, exact=True)
    hit = d > 0
    assert hit.mean() > 0.85
    # interior pixels (away from the fused region's border)
    inner = np.zeros_like(hit)
    inner[6:-6, 6:-6] = True
    sel = hit & inner
    assert np.abs(d[sel] - ex.depth[sel]).max() < 2e-6
    ang = np.arccos(np.clip(np.sum(n[sel] * ex.normals[sel], -1), -1, 1))
    assert ang.max() < 1e-4


def _sphere_scene():
    s = scenes.tiny_scene(1)
    s.noise_s0 = 0.0
    return s


def test_sphere_depth_within_discretisation_bound():
    """Curved surfaces: error bounded by O(h^2 / R) (trilinear + tangent-plane)."""
    s = _sphere_scene()
    P = oracle.Params(voxel_size=0.01, truncation=0.04, dense_dim=64)
    m = oracle.OracleMap(P)
    for i in range(10):
        f = s.frame(i)
        m.integrate(f.depth, f.rgb, s.K, f.pose)
    for fi in (3, 9):
        d, n, c, cok = m.render(s.K, s.poses[fi])
        ex = s.render(s.poses[fi], noise=False, exact=True)
        sph = (ex.ids == 2) & (d > 0)
        # ignore the silhouette ring
        interior = sph & (np.abs(np.sum(ex.normals * ex.points, -1)) /
                          np.maximum(np.linalg.norm(ex.points, axis=-1), 1e-9) > 0.5)
        if interior.sum() < 20:
            continue
        err = np.abs(d[interior] - ex.depth[interior])
        assert np.median(err) < 1e-3 and np.percentile(err, 95) < 4e-3


@pytest.mark.parametrize("fi", [1, 8])
def test_thin_plate_renders_the_visible_side(fi):
    """Lemma 1: seen from either side, the 5 mm plate renders its near face and
    never its far face."""
    s = _sphere_scene()
    P = oracle.Params(voxel_size=0.01, truncation=0.04, dense_dim=64)
    m = oracle.OracleMap(P)
    for i in range(10):
        f = s.frame(i)
        m.integrate(f.depth, f.rgb, s.K, f.pose)
    T = s.poses[fi]
    d, n, c, cok = m.render(s.K, T)
    ex = s.render(T, noise=False, exact=True)
    # hit points at least two voxels away from the plate's rim (the rim itself is an edge
    # where the directions' gradients mix)
    pw = ex.points @ T[:3, :3].T + T[:3, 3]
    c, e = s.prims[1, 2:5], s.prims[1, 5:8]
    rim = np.minimum(e[1] - np.abs(pw[..., 1] - c[1]), e[2] - np.abs(pw[..., 2] - c[2]))
    plate = (ex.ids == 1) & (d > 0) & (rim > 2 * P.voxel_size)
    assert plate.sum() > 300
    err = d[plate] - ex.depth[plate]
    # the far face lies >= 5 mm behind the near one along the view ray; the few pixels off
    # the near face hit spurious fused surfaces in front of it (err < 0), never the far face
    assert np.mean(np.abs(err) < 1e-3) > 0.98
    assert np.mean(err > 3e-3) < 0.002


def test_unobserved_space_is_a_miss():
    P = oracle.Params(voxel_size=0.01, truncation=0.04, dense_dim=64)
    m = oracle.OracleMap(P)
    s = scenes.tiny_scene(1)
    d, n, c, cok = m.render(s.K, s.poses[0])
    assert np.all(d == 0)
