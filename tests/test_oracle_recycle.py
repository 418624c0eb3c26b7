"""Pins of the oracle's voxel recycling (Sec. 3): the removed bricks are exactly those whose
weighted voxels are all at or above the free-space threshold, the kept bricks are untouched,
recycling commutes with later fusion for the kept bricks, and the render changes only next to the
removed bricks."""
import numpy as np

import oracle
import scenes

THR = 0.75


def _scene():
    s = scenes.tiny_scene(1)
    s.noise_s0 = 0.0
    return s


def _fused(s, frames):
    m = oracle.OracleMap(oracle.Params(voxel_size=0.01, truncation=0.04))
    for i in frames:
        f = s.frame(i)
        m.integrate(f.depth, f.rgb, s.K, f.pose)
    return m


def _snapshot(m):
    return {tuple(b[:4]): m.brick(*b[:4]).copy() for b in m.bricks()}


def test_recycle_removes_exactly_the_free_bricks():
    s = _scene()
    m = _fused(s, range(10))
    before = _snapshot(m)
    free = {k for k, v in before.items() if np.all((v[:, 1] <= 0) | (v[:, 0] >= THR))}
    assert len(free) > 20
    n = m.recycle(THR)
    after = _snapshot(m)
    assert n == len(free) and m.num_bricks() == len(before) - n
    assert set(after) == set(before) - free
    for k, v in after.items():
        assert np.array_equal(v, before[k])
    assert m.recycle(THR) == 0  # nothing left to remove


def test_recycling_commutes_with_later_fusion_for_kept_bricks():
    s = _scene()
    a = _fused(s, range(6))
    b = _fused(s, range(6))
    removed = a.recycle(THR)
    assert removed > 0
    for i in range(6, 10):
        f = s.frame(i)
        a.integrate(f.depth, f.rgb, s.K, f.pose)
        b.integrate(f.depth, f.rgb, s.K, f.pose)
    sa, sb = _snapshot(a), _snapshot(b)
    assert set(sa) <= set(sb)  # allocation depends on the frame alone
    same = 0
    for k, v in sa.items():
        if np.array_equal(v, sb[k]):
            same += 1
    # bricks re-created after removal restart from empty voxels; every other one is identical
    assert same >= len(sa) - removed


def test_render_changes_only_next_to_removed_bricks():
    """Removing free-space bricks changes the field only at samples whose trilinear corners or
    gradient taps reach into a removed brick: every pixel whose render changed hits within
    two voxels of a removed brick's cube, and the hit mask is unchanged."""
    s = _scene()
    m = _fused(s, range(10))
    T = s.poses[4] @ scenes.perturbation(np.random.default_rng(2), 1.0, 0.005)
    d0, n0, _, _ = m.render(s.K, T)
    before = {tuple(b[:4]) for b in m.bricks()}
    m.recycle(THR)
    removed = before - {tuple(b[:4]) for b in m.bricks()}
    d1, n1, _, _ = m.render(s.K, T)
    assert np.mean((d0 > 0) == (d1 > 0)) >= 0.999
    both = (d0 > 0) & (d1 > 0)
    changed = both & (d0 != d1)
    assert np.mean(changed[both]) < 0.01
    K, h = s.K, 0.01
    v, u = np.nonzero(changed)
    pts = np.stack([(u - K.cx) / K.fx, (v - K.cy) / K.fy, np.ones_like(u, float)], -1) * d0[v, u][:, None]
    pw = pts @ T[:3, :3].T + T[:3, 3]
    cubes = np.array(sorted({k[:3] for k in removed}), float) * 8 * h
    # distance from each changed hit to the nearest removed cube [c, c + 8h]^3
    dlo = np.maximum(cubes[None] - pw[:, None], 0.0)
    dhi = np.maximum(pw[:, None] - (cubes[None] + 8 * h), 0.0)
    dist = np.linalg.norm(np.maximum(dlo, dhi), axis=-1).min(1)
    assert dist.max() <= 2 * h, dist.max()
