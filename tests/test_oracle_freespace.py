"""Pins of the oracle's free-space combination render (Sec. 4, Alg. 1) on analytic scenes:
the same closed forms and the same Lemma 1 property as the direct render."""
import numpy as np
import pytest

import angles
import oracle
import scenes


def _fused(scene, n, **kw):
    P = oracle.Params(voxel_size=0.01, truncation=0.04, **kw)
    m = oracle.OracleMap(P)
    for i in range(n):
        f = scene.frame(i)
        m.integrate(f.depth, f.rgb, scene.K, f.pose)
    return m, P


def test_plane_render_is_exact():
    """One plane: a single direction takes part, its field is linear, so the render is the
    analytic ray-plane intersection and its normal."""
    s = scenes.plane_scene()
    m, _ = _fused(s, 4)
    T = s.poses[1].copy()
    T[:3, 3] += np.array([0.01, -0.02, 0.01])
    d, n = m.render_freespace(s.K, T)
    ex = s.render(T, noise=False, exact=True)
    hit = d > 0
    assert hit.mean() > 0.85
    inner = np.zeros_like(hit)
    inner[6:-6, 6:-6] = True
    sel = hit & inner
    # the float32 depth input bounds it (test_oracle_render.test_plane_render_is_exact)
    assert np.abs(d[sel] - ex.depth[sel]).max() < 5e-7
    ang = angles.between(n[sel], ex.normals[sel])
    assert ang.max() < 2e-5


def _tiny():
    s = scenes.tiny_scene(1)
    s.noise_s0 = 0.0
    return s


@pytest.mark.parametrize("fi", [1, 8])
def test_thin_plate_renders_the_visible_side(fi):
    """Lemma 1 with Alg. 1's free-space decision: the 5 mm plate renders its near face, never
    its far face (whose direction holds negative values in front of the near face)."""
    s = _tiny()
    m, P = _fused(s, 10, dense_dim=64)
    T = s.poses[fi]
    sub = np.stack(np.meshgrid(np.arange(0, s.K.width, 2), np.arange(0, s.K.height, 2)), -1).reshape(-1, 2)
    d, n = m.render_freespace(s.K, T, sub)
    ex = s.render(T, noise=False, exact=True)
    u, v = sub[:, 0], sub[:, 1]
    pw = ex.points[v, u] @ T[:3, :3].T + T[:3, 3]
    c, e = s.prims[1, 2:5], s.prims[1, 5:8]
    rim = np.minimum(e[1] - np.abs(pw[:, 1] - c[1]), e[2] - np.abs(pw[:, 2] - c[2]))
    plate = (ex.ids[v, u] == 1) & (d > 0) & (rim > 2 * P.voxel_size)
    assert plate.sum() > 80
    err = d[plate] - ex.depth[v, u][plate]
    assert np.mean(np.abs(err) < 1e-3) > 0.97
    assert np.mean(err > 3e-3) < 0.01


def test_sphere_depth_within_discretisation_bound():
    s = _tiny()
    m, _ = _fused(s, 10, dense_dim=64)
    seen = 0
    for fi in (3, 9):
        T = s.poses[fi]
        d, n = m.render_freespace(s.K, T)
        ex = s.render(T, noise=False, exact=True)
        sph = (ex.ids == 2) & (d > 0)
        interior = sph & (np.abs(np.sum(ex.normals * ex.points, -1)) /
                          np.maximum(np.linalg.norm(ex.points, axis=-1), 1e-9) > 0.5)
        if interior.sum() < 20:
            continue
        seen += 1
        err = np.abs(d[interior] - ex.depth[interior])
        assert np.median(err) < 1e-3 and np.percentile(err, 95) < 4e-3
    assert seen >= 1


def test_unobserved_space_is_a_miss():
    s = scenes.tiny_scene(1)
    m = oracle.OracleMap(oracle.Params(voxel_size=0.01, truncation=0.04, dense_dim=64))
    d, n = m.render_freespace(s.K, s.poses[0], np.array([[80, 60], [10, 10]]))
    assert np.all(d == 0)


def test_agrees_with_the_direct_render_away_from_conflicts():
    """On the box room (no thin structure in view of frame 3's centre), Alg. 1 and the weighting of
    Eq. combine_weight find the same surface: depths agree to discretisation error."""
    s = _tiny()
    m, _ = _fused(s, 10, dense_dim=64)
    T = s.poses[3]
    sub = np.stack(np.meshgrid(np.arange(40, 120, 3), np.arange(30, 90, 3)), -1).reshape(-1, 2)
    d1, _ = m.render_freespace(s.K, T, sub)
    d0, _, _, _ = m.render(s.K, T, sub)
    both = (d0 > 0) & (d1 > 0)
    assert both.mean() > 0.9
    assert np.median(np.abs(d1[both] - d0[both])) < 5e-4
