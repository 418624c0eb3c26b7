"""Pins of the oracle's preprocessing and fusion (Sec. 3, Sec. 7) on closed forms."""
import numpy as np
import pytest

import oracle
import scenes


def brute_filter(depth, zmin, zmax, dsup):
    H, W = depth.shape
    ok = np.zeros_like(depth, dtype=bool)
    for v in range(H):
        for u in range(W):
            z = depth[v, u]
            if not (z > 0 and zmin <= z <= zmax):
                continue
            c = 0
            for dv in (-1, 0, 1):
                for du in (-1, 0, 1):
                    if du == 0 and dv == 0:
                        continue
                    uu, vv = u + du, v + dv
                    if 0 <= uu < W and 0 <= vv < H:
                        zn = depth[vv, uu]
                        if zn > 0 and zmin <= zn <= zmax and abs(float(zn) - float(z)) <= dsup:
                            c += 1
            ok[v, u] = c >= 2
    return ok


def test_outlier_filter_brute_force():
    rng = np.random.default_rng(3)
    d = rng.uniform(0.5, 0.6, size=(15, 20)).astype(np.float32)
    d[rng.random(d.shape) < 0.2] = 0
    d[rng.random(d.shape) < 0.1] += 0.5
    K = scenes.Intrinsics(20, 15, 20.0, 20.0, 9.5, 7.0)
    out = oracle.preprocess(d, K, 0.1, 6.0, 0.01)
    assert np.array_equal(out["ok"].astype(bool), brute_filter(d, 0.1, 6.0, np.float32(0.01)))


def test_plane_normals_exact():
    s = scenes.plane_scene()
    f = s.frame(0, exact=True)
    out = oracle.preprocess(f.depth, s.K, 0.1, 6.0, 0.01)
    m = out["nok"].astype(bool)
    assert m.mean() > 0.9
    ang = np.arccos(np.clip(np.sum(out["n"][m] * f.normals[m], -1), -1, 1))
    assert ang.max() < 2e-4   # limited only by the float32 depth input


def _fuse_plane(times=1, color=True):
    s = scenes.plane_scene()
    P = oracle.Params(voxel_size=0.01, truncation=0.04, w_max=255.0)
    m = oracle.OracleMap(P)
    f = s.frame(0, exact=True)
    for _ in range(times):
        m.integrate(f.depth, f.rgb if color else None, s.K, f.pose)
    return s, P, m, f


def _voxel_centres(b):
    i = np.arange(512)
    loc = np.stack([i % 8, (i // 8) % 8, i // 64], -1)
    return (8 * np.asarray(b[:3]) + loc)


def test_single_frame_plane_sdf_weight_colour_closed_form():
    s, P, m, f = _fuse_plane()
    n_w = s.extra["normal"]
    off = s.extra["offset"]
    T = f.pose
    R, t = T[:3, :3], T[:3, 3]
    K = s.K
    checked = 0
    for b in m.bricks():
        data = m.brick(*b[:4])
        D = b[3]
        x = _voxel_centres(b) * P.voxel_size
        upd = data[:, 1] > 0
        if not upd.any():
            continue
        dist = x @ n_w - off                      # signed distance to the plane, + in front
        xc = (x - t) @ R
        uf = xc[:, 0] / xc[:, 2] * K.fx + K.cx
        vf = xc[:, 1] / xc[:, 2] * K.fy + K.cy
        # skip voxels whose association is a rounding tie or whose band test is a tie
        safe = (np.abs(uf - np.round(uf) - 0.5) > 1e-3) & (np.abs(np.abs(uf - np.round(uf)) - 0.5) > 1e-3)
        safe &= (np.abs(np.abs(vf - np.round(vf)) - 0.5) > 1e-3) & (np.abs(np.abs(dist) - P.truncation) > 1e-5)
        carved = dist > P.truncation
        band = upd & safe & ~carved
        # sdf: the clamped plane distance (Eq. point-to-plane, d > 0 in front)
        assert np.allclose(data[band, 0], np.clip(dist[band] / P.truncation, -1, 1), atol=1e-5)
        # carved voxels: value 1 with the constant carving weight
        cv = upd & safe & carved
        assert np.allclose(data[cv, 0], 1.0) and np.allclose(data[cv, 1], P.w_carve)
        # weight: w_depth * w_angle * w_dir (Eq. combined_fusion_weight) from the analytic geometry
        u = np.floor(uf[band] + 0.5).astype(int)
        v = np.floor(vf[band] + 0.5).astype(int)
        zpix = f.points[v, u, 2]
        ray = np.stack([(u - K.cx) / K.fx, (v - K.cy) / K.fy, np.ones_like(zpix)], -1)
        ray /= np.linalg.norm(ray, axis=1, keepdims=True)
        n_c = R.T @ n_w
        w_angle = -(ray @ n_c)
        cosD = n_w[D >> 1] * (1 if D % 2 == 0 else -1)
        w_dir = oracle.w_dir(cosD, P.theta)
        w_exp = (1.0 / (zpix + 1.0 - P.z_min) ** 2) * w_angle * w_dir
        assert np.allclose(data[band, 1], w_exp, rtol=1e-4)
        # colour: the associated pixel's colour, weight w_d (1 - ||p - x|| / tau) (Eq. color_weight)
        cw = data[band, 5] > 0
        assert np.allclose(data[band][cw, 2:5], f.rgb[v[cw], u[cw]].astype(np.float64), atol=1e-9)
        p_cam = f.points[v, u]
        dpx = np.linalg.norm(p_cam - xc[band], axis=1)
        wc_exp = w_exp * (1 - np.minimum(1, dpx / P.truncation))
        assert np.allclose(data[band, 5], wc_exp, rtol=1e-4, atol=1e-6)
        checked += band.sum()
    assert checked > 1000


def test_running_average_identity():
    _, P, m1, _ = _fuse_plane(1)
    _, _, m3, _ = _fuse_plane(3)
    b1 = {tuple(b[:4]): m1.brick(*b[:4]) for b in m1.bricks()}
    for b in m3.bricks():
        d3 = m3.brick(*b[:4])
        d1 = b1[tuple(b[:4])]
        upd = d1[:, 1] > 0
        assert np.allclose(d3[upd, 0], d1[upd, 0], atol=1e-12)
        assert np.allclose(d3[upd, 1], np.minimum(3 * d1[upd, 1], P.w_max), rtol=1e-12)
        assert np.allclose(d3[upd, 2:5], d1[upd, 2:5], atol=1e-9)


def test_constant_colour_scene_fuses_to_that_colour():
    s = scenes.tiny_scene(2)
    s.prims[:, 17:20] = (37, 150, 211)
    s.prims[:, 20:23] = (37, 150, 211)
    P = oracle.Params(voxel_size=0.01, truncation=0.04, dense_dim=64)
    m = oracle.OracleMap(P)
    for i in range(0, 10, 3):
        f = s.frame(i)
        m.integrate(f.depth, f.rgb, s.K, f.pose)
    total = 0
    for b in m.bricks()[:600]:
        d = m.brick(*b[:4])
        c = d[:, 5] > 0
        total += c.sum()
        assert np.allclose(d[c, 2:5], (37, 150, 211), atol=1e-9)
    assert total > 1000


def test_depth_noise_free_voxels_beyond_band_untouched():
    # voxels farther than tau behind the observed surface are never updated (Sec. 3)
    s, P, m, f = _fuse_plane()
    n_w, off = s.extra["normal"], s.extra["offset"]
    for b in m.bricks():
        d = m.brick(*b[:4])
        x = _voxel_centres(b) * P.voxel_size
        behind = (x @ n_w - off) < -P.truncation - 1e-4
        assert np.all(d[behind, 1] == 0)
