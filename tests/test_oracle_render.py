"""Pins of the oracle's ray-cast render (Sec. 4) on analytic scenes."""
import numpy as np
import pytest

import angles
import oracle
import scenes


def test_plane_render_is_exact():
    """A fused plane is a linear field; trilinear interpolation and the convex
    combination of directions reproduce it exactly, so the render equals the
    analytic ray-plane intersection up to the float32 depth input. That input is
    rounded to ~6e-8 m at 1-2 m; the pixel normals formed from it over two-pixel
    baselines carry ~2e-5 rad, and a fused sdf at up to tau from its point moves by
    that times the lever arm (<= 8e-7 m) before the running averages smooth it: the
    bounds are 5e-7 m in depth and 2e-5 rad in the normal (measured: 8.8e-8 m and
    3.4e-6 rad)."""
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
    assert np.abs(d[sel] - ex.depth[sel]).max() < 5e-7
    ang = angles.between(n[sel], ex.normals[sel])
    assert ang.max() < 2e-5


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
    # Lemma 1 (Sec. 4): the near face is rendered, never the far face (5 mm behind it along the
    # ray) nor a point displaced toward it. Every hit on the plate's pixels is the near face
    # (within 1 mm: the discretisation bound at 1 cm voxels) or a different surface more than tau
    # away: flying surfaces of the arc's frames in front of it, or, through holes of the fused
    # plate, the scene behind it (no more than 0.2 % of the pixels)
    near = np.abs(err) < 1e-3
    assert np.all(near | (np.abs(err) > P.truncation)), np.sort(err[~near])
    assert near.mean() > 0.985
    assert np.mean(err > P.truncation) < 0.002


def test_unobserved_space_is_a_miss():
    P = oracle.Params(voxel_size=0.01, truncation=0.04, dense_dim=64)
    m = oracle.OracleMap(P)
    s = scenes.tiny_scene(1)
    d, n, c, cok = m.render(s.K, s.poses[0])
    assert np.all(d == 0)


def _coloured_plane_scene(colA, colB):
    """scenes.plane_scene's slab split in two along its first in-plane axis: one half of constant
    colour colA, the other of constant colour colB (top faces coplanar)."""
    s = scenes.plane_scene()
    p = s.prims[0]
    R = p[8:17].reshape(3, 3)
    a = R[0]
    left, right = p.copy(), p.copy()
    left[2:5] = p[2:5] - 1.5 * a
    right[2:5] = p[2:5] + 1.5 * a
    left[5] = right[5] = 1.5
    left[17:20] = left[20:23] = colA
    right[17:20] = right[20:23] = colB
    s.prims = np.stack([left, right])
    s.extra["split_axis"] = a
    return s


def _fused_colour_plane(colA, colB):
    s = _coloured_plane_scene(colA, colB)
    P = oracle.Params(voxel_size=0.01, truncation=0.04)
    m = oracle.OracleMap(P)
    for i in range(4):
        f = s.frame(i)
        m.integrate(f.depth, f.rgb, s.K, f.pose)
    T = s.poses[1].copy()
    T[:3, 3] += np.array([0.01, -0.02, 0.01])
    return s, P, m, T


def test_constant_colour_plane_renders_that_colour():
    """Eq. color_weight and the colour output of Sec. 4: every voxel of a constant-colour surface
    holds that colour, so every convex combination of them (trilinear, then over directions)
    renders exactly it."""
    col = (37, 150, 211)
    s, P, m, T = _fused_colour_plane(col, col)
    d, n, c, cok = m.render(s.K, T)
    hit = d > 0
    assert hit.mean() > 0.85 and cok[hit].mean() > 0.8
    sel = cok > 0
    assert np.abs(c[sel] - np.array(col, float)).max() < 1e-9


def test_two_colour_plane_renders_each_side_and_mixes_only_at_the_seam():
    """Two coplanar halves of constant colours A and B: a hit farther than tau + 2 voxels from
    the seam renders exactly its side's colour (colour is fused only within tau of the observed
    point, the trilinear corners and direction sum reach one voxel further); every rendered
    colour lies on the segment from A to B (a dropped weight or swapped channel leaves it)."""
    A, B = np.array((200.0, 30.0, 90.0)), np.array((10.0, 220.0, 140.0))
    s, P, m, T = _fused_colour_plane(A, B)
    d, n, c, cok = m.render(s.K, T)
    sel = cok > 0
    assert sel.mean() > 0.8
    K = s.K
    v, u = np.nonzero(sel)
    pts = np.stack([(u - K.cx) / K.fx, (v - K.cy) / K.fy, np.ones_like(u, float)], -1) * d[v, u][:, None]
    side = (pts @ T[:3, :3].T + T[:3, 3]) @ s.extra["split_axis"]
    far = P.truncation + 2 * P.voxel_size
    ca, cb = c[v, u][side < -far], c[v, u][side > far]
    assert len(ca) > 300 and len(cb) > 300
    assert np.abs(ca - A).max() < 1e-9 and np.abs(cb - B).max() < 1e-9
    # on the segment A-B: c = A + s (B - A), 0 <= s <= 1, nothing orthogonal to it
    AB = B - A
    x = c[v, u] - A
    sp = x @ AB / (AB @ AB)
    assert sp.min() > -1e-9 and sp.max() < 1 + 1e-9
    assert np.abs(x - sp[:, None] * AB).max() < 1e-9
    mixed = (sp > 1e-6) & (sp < 1 - 1e-6)
    assert mixed.any() and np.abs(side[mixed]).max() <= far
