"""Pins of the oracle's block allocation (Sec. 7) against a brute-force slab test."""
import itertools

import numpy as np

import oracle
import scenes


def slab_blocks(a, b, bs, origin=(0, 0, 0)):
    """All blocks whose cube [k bs, (k+1) bs) meets segment a-b, by exact FP64 slab tests."""
    a = np.asarray(a, np.float64) - origin
    b = np.asarray(b, np.float64) - origin
    lo = np.floor(np.minimum(a, b) / bs).astype(int) - 1
    hi = np.floor(np.maximum(a, b) / bs).astype(int) + 1
    d = b - a
    out = set()
    for c in itertools.product(*[range(lo[k], hi[k] + 1) for k in range(3)]):
        t0, t1 = 0.0, 1.0
        ok = True
        for k in range(3):
            bl, bh = c[k] * bs, (c[k] + 1) * bs
            if d[k] == 0:
                if not (bl <= a[k] < bh):
                    ok = False
                    break
                continue
            u0, u1 = (bl - a[k]) / d[k], (bh - a[k]) / d[k]
            t0, t1 = max(t0, min(u0, u1)), min(t1, max(u0, u1))
        if ok and t0 <= t1:
            out.add(tuple(c))
    return out


def boundary_distance(a, b, bs):
    """Smallest distance of the segment's points (sampled densely) to a block face plane."""
    ts = np.linspace(0, 1, 2001)[:, None]
    p = np.asarray(a) + ts * (np.asarray(b) - np.asarray(a))
    r = np.abs(p / bs - np.round(p / bs)) * bs
    return float(r.min())


def test_segment_blocks_match_brute_force():
    rng = np.random.default_rng(1)
    bs = np.float32(0.04)
    mism = 0
    for _ in range(3000):
        a = rng.uniform(-1, 1, 3).astype(np.float32)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        b = (a + rng.uniform(0.0, 0.12) * d).astype(np.float32)
        got = {tuple(c) for c in oracle.segment_blocks(a, b, bs)}
        exp = slab_blocks(a.astype(np.float64), b.astype(np.float64), float(bs))
        if got != exp:
            # only admissible where the segment grazes a block boundary within float rounding
            assert boundary_distance(a, b, float(bs)) < 1e-5, (a, b, got, exp)
            mism += 1
    assert mism <= 3


def test_axis_parallel_and_degenerate_segments():
    bs = np.float32(0.04)
    a = np.array([0.01, 0.01, 0.01], np.float32)
    assert {tuple(c) for c in oracle.segment_blocks(a, a, bs)} == {(0, 0, 0)}
    b = np.array([0.13, 0.01, 0.01], np.float32)
    assert {tuple(c) for c in oracle.segment_blocks(a, b, bs)} == {(0, 0, 0), (1, 0, 0), (2, 0, 0), (3, 0, 0)}
    c = np.array([0.01, -0.05, 0.01], np.float32)
    assert {tuple(x) for x in oracle.segment_blocks(a, c, bs)} == {(0, 0, 0), (0, -1, 0), (0, -2, 0)}


def test_frame_allocation_is_union_of_pixel_segments():
    """The bricks allocated by one frame equal the union over pixels with a normal of
    (slab-test blocks of [p - tau r, p + tau r]) x (directions the normal belongs to)."""
    s = scenes.planes_scene()
    K = scenes.Intrinsics(40, 30, 30.0, 30.0, 19.5, 14.5)
    f = s.render(s.poses[0], K=K, noise=False)
    P = oracle.Params(voxel_size=0.02, truncation=0.08)
    m = oracle.OracleMap(P)
    m.integrate(f.depth, f.rgb, K, f.pose)
    got = {tuple(b[:4]) for b in m.bricks()}
    pre = oracle.preprocess(f.depth, K, P.z_min, P.z_max, P.delta_sup)
    R = f.pose[:3, :3]
    t = f.pose[:3, 3]
    expected = set()
    graze = 0
    cos_t = np.cos(P.theta)
    bs = 8 * P.voxel_size
    for v in range(K.height):
        for u in range(K.width):
            if not pre["nok"][v, u]:
                continue
            nw = R @ pre["nd"][v, u]
            dirs = [D for D in range(6) if (nw[D >> 1] if D % 2 == 0 else -nw[D >> 1]) > cos_t]
            rv = R @ pre["Pd"][v, u]
            p = rv + t
            rh = rv / np.linalg.norm(rv)
            a, b = p - P.truncation * rh, p + P.truncation * rh
            for c in slab_blocks(a, b, bs):
                for D in dirs:
                    expected.add((*c, D))
            graze += boundary_distance(a, b, bs) < 1e-5
    diff = got ^ expected
    assert len(diff) <= 2 * graze + 2, (len(diff), graze)
    assert len(got) > 50
