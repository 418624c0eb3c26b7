"""Parity at the benchmark's full size: the 640x480 Kinect-shaped room (5 mm voxels, tau 2 cm,
colour), the renderer in the launch configuration bench.py times (default render options), the
coarse-to-fine schedules the benchmark runs, and fusion from scratch.

The oracle fuses 30 of the 300 frames in FP64. For the renderer alone its map, rounded to FP32,
is loaded into a device map (dtsdf_map_import), so the render is compared on identical voxels;
end to end, the device fuses the same 30 frames itself (the apron push and brick-bound
maintenance of the fusion kernels at scale) and its map is compared voxel by voxel with the
oracle's, up to the oracle's ties (tests/mapcheck.py), then rendered. The oracle renders a
regular sample of the pixels (every 4th row and column, 19,200 rays per pose) for the render
checks and the whole frame for the registrations. Tolerances (the benchmark spec): depth <= 1e-4 m and
normals <= 1e-3 rad on >= 99.9 % of the pixels both sides hit, hit-mask agreement >= 99.9 %,
pose <= 1e-4 rad / 1e-4 m. Both sides evaluate the normal at the root of the crossing (reading
C7), the oracle's root by bisection to 1e-10 m, the device's by 12 bisection steps and a linear
root of the last bracket (< 1 um). The FP16 storage form is held to its own bars (depth within
1e-4 m on >= 99.9 % of the jointly hit pixels, normals within 1e-3 rad on >= 99 %)."""
import numpy as np
import pytest

import angles
import oracle
from oracle import icp as oicp
import scenes
from mapcheck import SDF_TOL, W_ABS, W_REL, compare_maps

torch = pytest.importorskip("torch")
import paper_2301_12796_gb300 as dt  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
KW = dict(voxel_size=0.005, truncation=0.02, color=True)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def full():
    s = scenes.kinect_room(1)
    om = oracle.OracleMap(oracle.Params(z_max=s.z_max, **KW))
    for i in range(0, 300, 10):
        f = s.frame(i)
        om.integrate(f.depth, f.rgb, s.K, f.pose)
    ob = om.bricks()
    vox = np.stack([om.brick(*b[:4]) for b in ob]).astype(np.float32)
    gm = dt.Map(dt.params(max_blocks=len(ob) + 64, z_max=s.z_max, **KW))
    gm.import_bricks(ob[:, :4], vox)
    torch.cuda.synchronize()
    yield s, om, gm
    gm.close()


def render_gpu(gm, K, T):
    d = torch.zeros(K.height, K.width, device=DEV)
    n = torch.zeros(K.height, K.width, 4, device=DEV)
    c = torch.zeros(K.height, K.width, 4, device=DEV)
    gm.render(K, T, d, n, c)
    torch.cuda.synchronize()
    return d.cpu().numpy(), n.cpu().numpy(), c.cpu().numpy()


@pytest.mark.parametrize("fi", [20, 150, 280])
def test_full_size_render_matches_oracle_on_sampled_pixels(full, fi):
    s, om, gm = full
    K = s.K
    T = s.poses[fi]
    dg, ng, cg = render_gpu(gm, K, T)
    vv, uu = np.mgrid[0:K.height:4, 0:K.width:4]
    pix = np.stack([uu.ravel(), vv.ravel()], 1).astype(np.int32)
    do, no, co, cok = om.render(K, T, pix)
    g_d = dg[pix[:, 1], pix[:, 0]]
    g_n = ng[pix[:, 1], pix[:, 0], :3]
    g_c = cg[pix[:, 1], pix[:, 0]]
    hg, ho = g_d > 0, do > 0
    agree = np.mean(hg == ho)
    both = hg & ho
    assert both.sum() > 10000
    derr = np.abs(g_d[both] - do[both])
    nerr = angles.between(g_n[both], no[both])
    print(f"pose {fi}: mask {agree:.5f} depth<=1e-4 {np.mean(derr <= 1e-4):.5f} median {np.median(derr):.2e} "
          f"normals<=1e-3 {np.mean(nerr <= 1e-3):.5f} max {nerr.max():.2e}")
    assert agree >= 0.999, agree
    assert np.mean(derr <= 1e-4) >= 0.999, np.mean(derr <= 1e-4)
    assert np.mean(nerr <= 1e-3) >= 0.999, np.mean(nerr <= 1e-3)
    close = both & (g_c[:, 3] > 0) & (cok > 0)
    close[both] &= derr <= 1e-4
    assert np.quantile(np.abs(g_c[close][:, :3] - co[close]).max(-1), 0.999) <= 0.5


def test_full_size_registration_matches_oracle(full):
    s, om, gm = full
    K = s.K
    T_ref = s.poses[150]
    cur = s.frame(152)
    # device: render at the reference pose, then the whole schedule on the device
    d = torch.zeros(K.height, K.width, device=DEV)
    n = torch.zeros(K.height, K.width, 4, device=DEV)
    gm.render(K, T_ref, d, n)
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_frame(cu(cur.depth), None, K, 0.1, s.z_max, 0.01)
    opts = dt.icp_opts(levels=3, iters=(10, 5, 4), eps=(0.005, 0.05, 0.05), lam=0.0)
    Tdev = torch.eye(4, dtype=torch.float64, device=DEV)
    ic.solve(d, n, K, Tdev, opts)
    Tg = Tdev.cpu().numpy()
    ic.close()
    # oracle: its own render of the whole frame, its own schedule
    do, no, _, _ = om.render(K, T_ref)
    rn = np.zeros(no.shape[:2] + (4,), np.float32)
    rn[..., :3] = no
    rn[..., 3] = do
    pre = oracle.preprocess(cur.depth, K, 0.1, s.z_max, 0.01)
    levels = oicp.pyramid(pre["z"], K, 3)
    st = oicp.Settings(eps=(0.005, 0.05, 0.05), iters=(10, 5, 4))
    To, _ = oicp.track(levels, do.astype(np.float32), rn, K, np.eye(4), st)
    ang = np.arccos(np.clip((np.trace(Tg[:3, :3].T @ To[:3, :3]) - 1) / 2, -1, 1))
    print(f"registration: device vs oracle {ang:.2e} rad, {np.linalg.norm(Tg[:3, 3] - To[:3, 3]):.2e} m")
    assert ang <= 1e-4 and np.linalg.norm(Tg[:3, 3] - To[:3, 3]) <= 1e-4
    # and the motion found is the true one to the noise level
    true = np.linalg.inv(T_ref) @ cur.pose
    assert np.linalg.norm(To[:3, 3] - true[:3, 3]) < 5e-3


KINECT_OPTS = dict(levels=3, iters=(10, 5, 4), eps=(0.005, 0.05, 0.05), photo_thr=(0.05, 0.175, 0.175), lam=0.1,
                   z_min=0.1, stop_norm=1e-6, min_rows=10)


def test_full_size_f2kf_schedule_matches_oracle(full):
    """The schedule the benchmark times: SE(3) point-to-plane plus frame-to-keyframe photometric
    rows (lambda 0.1, keyframe = the last frame whose index is a multiple of 10, render at the
    previous frame's pose), 3 levels 4/5/10 iterations, against the oracle's schedule on its
    own render of the same map."""
    s, om, gm = full
    K = s.K
    f = 152
    T_ref, T_kf = s.poses[f - 1], s.poses[150]
    cur, kf = s.frame(f), s.frame(150)
    T_rs = np.linalg.inv(T_kf) @ T_ref
    d = torch.zeros(K.height, K.width, device=DEV)
    n = torch.zeros(K.height, K.width, 4, device=DEV)
    gm.render(K, T_ref, d, n)
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_frame(cu(cur.depth), cu(cur.rgb), K, 0.1, s.z_max, 0.01)
    ic.set_keyframe(cu(kf.rgb), K)
    Tdev = torch.eye(4, dtype=torch.float64, device=DEV)
    Trs_dev = torch.from_numpy(T_rs).to(DEV)
    ic.solve(d, n, K, Tdev, dt.icp_opts(**KINECT_OPTS), T_rs_dev=Trs_dev)
    Tg = Tdev.cpu().numpy()
    ic.close()
    do, no, _, _ = om.render(K, T_ref)
    rn = np.zeros(no.shape[:2] + (4,), np.float32)
    rn[..., :3] = no
    rn[..., 3] = do
    pre = oracle.preprocess(cur.depth, K, 0.1, s.z_max, 0.01)
    levels = oicp.pyramid(pre["z"], K, 3, cur.rgb)
    kI = oicp.pyramid(pre["z"], K, 3, kf.rgb)
    photo = [(kI[l].I, K.scaled(l), T_rs) for l in range(3)]
    st = oicp.Settings(eps=(0.005, 0.05, 0.05), iters=(10, 5, 4), photo_thr=(0.05, 0.175, 0.175), lam=0.1)
    To, _ = oicp.track(levels, do.astype(np.float32), rn, K, np.eye(4), st, photo)
    ang = np.arccos(np.clip((np.trace(Tg[:3, :3].T @ To[:3, :3]) - 1) / 2, -1, 1))
    print(f"f2kf registration: device vs oracle {ang:.2e} rad, {np.linalg.norm(Tg[:3, 3] - To[:3, 3]):.2e} m")
    assert ang <= 1e-4 and np.linalg.norm(Tg[:3, 3] - To[:3, 3]) <= 1e-4
    true = np.linalg.inv(T_ref) @ cur.pose
    assert np.linalg.norm(To[:3, 3] - true[:3, 3]) < 5e-3


@pytest.fixture(scope="module")
def fused(full):
    """The device fuses the oracle's 30 frames itself (FP32 and FP16 storage)."""
    s, om, _ = full
    maps = {}
    for name, storage in (("fp32", dt.STORE_FP32), ("fp16", dt.STORE_FP16)):
        gm = dt.Map(dt.params(max_blocks=1 << 18, z_max=s.z_max, storage=storage, **KW))
        for i in range(0, 300, 10):
            f = s.frame(i)
            gm.integrate(cu(f.depth), cu(f.rgb), s.K, f.pose)
        maps[name] = gm
    torch.cuda.synchronize()
    yield maps
    for gm in maps.values():
        gm.close()


def test_full_size_fusion_matches_oracle(full, fused):
    s, om, _ = full
    r = compare_maps(fused["fp32"], om)
    print(f"full-size fusion: {r['checked']} voxels in {r['bricks']} bricks checked; differing on ties: "
          f"{r['tie_keys']} keys, {r['tie_voxels']} voxels, {r['tie_colour']} colours")
    assert r["checked"] > 10_000_000


def _sampled(gm, om, K, T):
    dg, ng, cg = render_gpu(gm, K, T)
    vv, uu = np.mgrid[0:K.height:4, 0:K.width:4]
    pix = np.stack([uu.ravel(), vv.ravel()], 1).astype(np.int32)
    do, no, co, cok = om.render(K, T, pix)
    g_d = dg[pix[:, 1], pix[:, 0]]
    g_n = ng[pix[:, 1], pix[:, 0], :3]
    hg, ho = g_d > 0, do > 0
    both = hg & ho
    derr = np.abs(g_d[both] - do[both])
    nerr = angles.between(g_n[both], no[both])
    return np.mean(hg == ho), derr, nerr, both.sum()


def _differing_voxels(gm, om):
    """World voxel coordinates (any direction) where the device-fused and the oracle-fused maps
    differ beyond the fusion tolerances: the voxels of bricks present on one side only, and the
    voxels whose presence, sdf or weight differ (all of them on the oracle's ties)."""
    coords, vox = gm.export()
    gidx = {tuple(int(x) for x in c): i for i, c in enumerate(coords)}
    oc, ov, _ = om.export()
    ijk = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1)
    ijk = ijk.transpose(2, 1, 0, 3).reshape(512, 3)  # voxel index i + 8 j + 64 k -> (i, j, k)
    out = []
    seen = set()
    for c, o in zip(oc, ov):
        key = tuple(int(x) for x in c)
        seen.add(key)
        base = 8 * np.array(key[:3])
        if key not in gidx:
            out.append(base + ijk)
            continue
        g = vox[gidx[key]].astype(np.float64)
        bad = (g[:, 1] > 0) != (o[:, 1] > 0)
        both = (g[:, 1] > 0) & (o[:, 1] > 0)
        bad[both] |= np.abs(g[both, 0] - o[both, 0]) > SDF_TOL
        bad[both] |= np.abs(g[both, 1] - o[both, 1]) > W_REL * o[both, 1] + W_ABS
        if bad.any():
            out.append(base + ijk[bad])
    for key, i in gidx.items():
        if key not in seen:
            out.append(8 * np.array(key[:3]) + ijk)
    return {tuple(v) for v in np.concatenate(out)} if out else set()


def _near_differing(K, T, pix, depth, h, differ):
    """Per hit pixel: whether the voxels its hit reads (trilinear corners and gradient taps: the
    4^3 voxels from the base corner - 1 to + 2) include one where the maps differ."""
    out = np.zeros(len(pix), bool)
    R, o = T[:3, :3], T[:3, 3]
    for i, ((u, v), d) in enumerate(zip(pix, depth)):
        rc = np.array([(u - K.cx) / K.fx, (v - K.cy) / K.fy, 1.0])
        x = o + d * (R @ rc)
        b = np.floor(x / h).astype(int)
        out[i] = any((b[0] + a, b[1] + bb, b[2] + c) in differ
                     for a in range(-1, 3) for bb in range(-1, 3) for c in range(-1, 3))
    return out


@pytest.fixture(scope="module")
def fused_in_oracle(full, fused):
    """The device-fused FP32 map loaded into an oracle map (the device's values, exactly)."""
    s, _, _ = full
    coords, vox = fused["fp32"].export()
    og = oracle.OracleMap(oracle.Params(z_max=s.z_max, **KW))
    for c, v in zip(coords, vox):
        og.set_brick(*c, v)
    return og


@pytest.fixture(scope="module")
def fused_differ(full, fused):
    return _differing_voxels(fused["fp32"], full[1])


@pytest.mark.parametrize("fi", [20, 150, 280])
def test_full_size_fused_map_renders_like_oracle(full, fused, fused_in_oracle, fused_differ, fi):
    """End to end at full size, in two parts.

    The renderer on the map the device fused: its render against the oracle's render of the same
    map (the device's values loaded into the oracle), at the renderer's bars (mask and depth on
    99.9 %, normals within 1e-3 rad on 99.9 %).

    The fusion's effect on the render: the oracle's renders of the device-fused map and of its own
    map differ only through the maps, which agree within the fusion tolerances except on voxels
    the oracle records as ties (its FP64 decision within FP32 rounding of the threshold), where
    one side updated a voxel and the other did not. Mask and depth are held on 99.9 %; the
    normal within 1e-3 rad on 99.9 % of the pixels whose hit reads no such voxel (the rest are
    counted)."""
    s, om, _ = full
    og = fused_in_oracle
    K, T = s.K, s.poses[fi]
    agree, derr, nerr, n = _sampled(fused["fp32"], og, K, T)
    print(f"fused pose {fi}, renderer: mask {agree:.5f} depth<=1e-4 {np.mean(derr <= 1e-4):.5f} "
          f"normals<=1e-3 {np.mean(nerr <= 1e-3):.5f} max {nerr.max():.2e}")
    assert n > 10000 and agree >= 0.999
    assert np.mean(derr <= 1e-4) >= 0.999 and np.mean(nerr <= 1e-3) >= 0.999
    vv, uu = np.mgrid[0:K.height:4, 0:K.width:4]
    pix = np.stack([uu.ravel(), vv.ravel()], 1).astype(np.int32)
    d1, n1, _, _ = og.render(K, T, pix)
    d0, n0, _, _ = om.render(K, T, pix)
    both = (d1 > 0) & (d0 > 0)
    agree = np.mean((d1 > 0) == (d0 > 0))
    derr = np.abs(d1[both] - d0[both])
    nerr = angles.between(n1[both], n0[both])
    near = _near_differing(K, T, pix[both], d0[both], 0.005, fused_differ)
    print(f"fused pose {fi}, maps: mask {agree:.5f} depth<=1e-4 {np.mean(derr <= 1e-4):.5f} normals<=1e-3 "
          f"{np.mean(nerr <= 1e-3):.5f}, off tie voxels {np.mean(nerr[~near] <= 1e-3):.5f} "
          f"({np.mean(near):.4f} of the hits read a tie voxel)")
    assert agree >= 0.999 and np.mean(derr <= 1e-4) >= 0.999
    assert np.mean(nerr[~near] <= 1e-3) >= 0.999


def test_full_size_fp16_map_matches_oracle(full, fused):
    """FP16 sdf, half weight, u8 colour at full size: allocation and presence equal to the
    oracle's up to its ties, sdf within the storage quantisation carried through the running
    averages, and the render on sampled pixels at the FP16 bars."""
    s, om, _ = full
    gm = fused["fp16"]
    coords, vox = gm.export()
    gidx = {tuple(c): i for i, c in enumerate(coords)}
    oc, ov, ot = om.export()
    errs = []
    for c, o, t in zip(oc, ov, ot):
        key = tuple(int(x) for x in c)
        if key not in gidx:
            assert om.alloc_tie(*key) >= 0
            continue
        g = vox[gidx[key]].astype(np.float64)
        tie = (t & 1) > 0
        assert np.all(((g[:, 1] > 0) == (o[:, 1] > 0)) | tie)
        p = (g[:, 1] > 0) & (o[:, 1] > 0) & ~tie
        if p.any():
            errs.append(np.abs(g[p, 0] - o[p, 0]))
            assert np.all(np.abs(g[p, 1] - o[p, 1]) <= 0.01 * o[p, 1] + 1e-5)
    e = np.concatenate(errs)
    print(f"fp16 full size: {e.size} voxels, sdf error q999 {np.quantile(e, 0.999):.2e} max {e.max():.2e}")
    assert np.quantile(e, 0.999) <= 2e-3 and e.max() <= 0.05
    agree, derr, nerr, n = _sampled(gm, om, s.K, s.poses[150])
    print(f"fp16 render: mask {agree:.5f} depth<=1e-4 {np.mean(derr <= 1e-4):.5f} normals {np.mean(nerr <= 1e-3):.5f}")
    assert agree >= 0.999 and np.mean(derr <= 1e-4) >= 0.999 and np.mean(nerr <= 1e-3) >= 0.99
