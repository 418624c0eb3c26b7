"""Pins of the oracle's view-dependent combined TSDF and its ray-cast (Sec. 4; Sec. 7: the
combination at integer voxel positions with 6-neighbour gradients)."""
import numpy as np

import angles
import oracle
import scenes

H = 0.01
TAU = 0.04
XP, XM = 0, 1  # directions X+ and X-


def _params():
    return oracle.Params(voxel_size=H, truncation=TAU, color=True)


def _linear_brick(block, grad, offset, w=1.0, rgb=(0.0, 0.0, 0.0)):
    """512 x 6 voxels of the linear field sdf = (grad . x_voxel + offset) / tau (voxel centres
    at (8 b + (i, j, k)) h), clamped to [-1, 1], weight w, colour rgb with colour weight w."""
    vi = np.arange(512)  # voxel index i + 8 j + 64 k
    xi, yi, zi = vi % 8, (vi // 8) % 8, vi // 64
    xw = ((8 * block[0] + xi) * H, (8 * block[1] + yi) * H, (8 * block[2] + zi) * H)
    sdf = np.clip((grad[0] * xw[0] + grad[1] * xw[1] + grad[2] * xw[2] + offset) / TAU, -1.0, 1.0)
    out = np.zeros((512, 6))
    out[:, 0] = sdf
    out[:, 1] = w
    out[:, 2:5] = rgb
    out[:, 5] = w
    return out


def _two_sided_map():
    """Blocks (-1..1)^3 of X+ holding a field rising along +x and of X- one rising along -x,
    both zero at x = 0.1 m, with different colours."""
    m = oracle.OracleMap(_params())
    for bx in range(-1, 2):
        for by in range(-1, 2):
            for bz in range(-1, 2):
                b = (bx, by, bz)
                m.set_brick(*b, XP, _linear_brick(b, (1.0, 0.0, 0.0), -0.1, w=2.0, rgb=(200.0, 10.0, 10.0)))
                m.set_brick(*b, XM, _linear_brick(b, (-1.0, 0.0, 0.0), 0.1, w=3.0, rgb=(10.0, 10.0, 200.0)))
    return m


def test_only_the_direction_facing_the_camera_contributes():
    """The normal of X+ points along +x, that of X- along -x; with the camera on the +x side only
    X+ faces the view ray (<n, -r> > 0), on the -x side only X-: the combined value and colour
    are those of one direction alone, whichever side the camera is on."""
    m = _two_sided_map()
    v = (9, 2, 3)  # |sdf| < 1 here and all 6 neighbours present in both directions
    x = v[0] * H
    for cam, want, col in (((5.0, 0.02, 0.03), (x - 0.1) / TAU, (200.0, 10.0, 10.0)),
                           ((-5.0, 0.02, 0.03), (0.1 - x) / TAU, (10.0, 10.0, 200.0))):
        ok, phi, rgb, cok = m.comb_voxel(*v, np.array(cam))
        assert ok and cok
        assert abs(phi - want) < 1e-12, (cam, phi, want)
        assert np.allclose(rgb, col, atol=1e-9)


def test_fallback_weights_without_gradients():
    """A voxel whose neighbours are missing has no gradient in any direction: the fallback
    weight W^D max(0, <v^D, -r>) of Eq. combine_tsdf_weight picks the direction whose axis faces
    the camera, and no colour is defined."""
    m = _two_sided_map()
    v = (15, 2, 3)  # x = 15: its +x neighbour (block 2) is not allocated
    for cam, D_sign in (((5.0, 0.02, 0.03), 1.0), ((-5.0, 0.02, 0.03), -1.0)):
        ok, phi, rgb, cok = m.comb_voxel(*v, np.array(cam))
        assert ok and not cok
        assert abs(phi - np.clip(D_sign * (v[0] * H - 0.1) / TAU, -1, 1)) < 1e-12


def test_identical_directions_combine_to_their_common_value():
    """Any convex combination of equal values is that value, whatever the weights."""
    m = oracle.OracleMap(_params())
    for bx in range(-1, 2):
        for by in range(-1, 2):
            for bz in range(-1, 2):
                b = (bx, by, bz)
                for D, w in ((0, 1.0), (2, 0.5), (4, 2.0)):
                    m.set_brick(*b, D, _linear_brick(b, (0.6, 0.48, 0.64), -0.02, w=w))
    rng = np.random.default_rng(1)
    for _ in range(20):
        v = rng.integers(-7, 14, size=3)
        cam = rng.normal(size=3) * 3
        ok, phi, _, _ = m.comb_voxel(*v, cam)
        want = np.clip((0.6 * v[0] * H + 0.48 * v[1] * H + 0.64 * v[2] * H - 0.02) / TAU, -1, 1)
        if ok:
            assert abs(phi - want) < 1e-12


def test_combined_plane_render_is_exact():
    """A fused plane is a linear field in every direction that stores it; its combination keeps
    the field, so the combined ray-cast from the pose of the combination equals the analytic
    ray-plane intersection (as the direct render does)."""
    s = scenes.plane_scene()
    m = oracle.OracleMap(oracle.Params(voxel_size=0.01, truncation=0.04))
    for i in range(4):
        f = s.frame(i)
        m.integrate(f.depth, f.rgb, s.K, f.pose)
    T = s.poses[1].copy()
    T[:3, 3] += np.array([0.01, -0.02, 0.01])
    m.combine(T[:3, 3])
    d, n, c, cok = m.render_combined(s.K, T)
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


def test_direction_weight_excludes_normals_far_from_the_axis():
    """Eq. direction_weight: a direction whose normal makes more than theta (3 pi / 8) with its
    axis gets no weight. X+ and Y+ both store fields rising along +y (normal +y), with different
    offsets; the normal is 90 degrees from the X+ axis, so only Y+ contributes."""
    m = oracle.OracleMap(_params())
    for bx in range(-1, 2):
        for by in range(-1, 2):
            for bz in range(-1, 2):
                b = (bx, by, bz)
                m.set_brick(*b, 0, _linear_brick(b, (0.0, 1.0, 0.0), -0.10, w=5.0))
                m.set_brick(*b, 2, _linear_brick(b, (0.0, 1.0, 0.0), -0.11, w=1.0))
    v = (2, 10, 3)  # y = 0.10: |sdf| < 1 in both directions
    ok, phi, _, _ = m.comb_voxel(*v, np.array([0.02, 5.0, 0.03]))
    assert ok and abs(phi - (v[1] * H - 0.11) / TAU) < 1e-12
