"""GPU-vs-oracle parity of fusion, rendering and ICP through the C ABI.

Tolerances (the required values where they exist, otherwise derived from the arithmetic below):
  render depth |d| <= 1e-4 m on pixels both sides hit, hit-mask agreement >= 99.9 %,
  normal angle <= 1e-3 rad; ICP pose <= 1e-4 rad / 1e-4 m / 1e-5 relative scale.
  The render is checked twice: on the oracle's own map loaded into the device map
  (renderer alone) and end to end after fusing on both sides (the FP32 map differs from
  the FP64 one by micrometres). The normal is a derivative of the map and jumps where a
  direction enters or leaves the combination, so like the hit mask it is held to its
  tolerance on >= 99.9 % of the pixels both sides hit; the largest deviation is bounded
  separately.
  fused voxels: FP32 running averages vs FP64: sdf |d| <= 2e-4 (units of tau), weights
  |d| <= 1e-4 w + 1e-5, colour |d| <= 1e-2 (0..255). The oracle decides every allocation and
  voxel update in FP64 and records its ties (decisions within the FP32 rounding of their
  thresholds); the allocated (block, D) sets, the voxels with weight > 0 and the voxel values
  may differ only on those (tests/mapcheck.py), and the counts of such differences are printed.
  ICP: the row counts may differ by at most the oracle's tie pixels, H and g by at most the
  bound on their other outcomes (oracle.icp.tie_bounds) on top of the arithmetic tolerance.
"""
import numpy as np
import pytest
import torch

import angles
import oracle
from oracle import icp as oicp
import scenes
from mapcheck import compare_maps as _compare
import paper_2301_12796_gb300 as dt
from paper_2301_12796_gb300 import build as B

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

DEPTH_TOL = 1e-4
MASK_AGREE = 0.999
NORMAL_TOL = 1e-3
# FP16 storage form: share of mask-agreeing pixels whose depth is within DEPTH_TOL
FP16_DEPTH_FRAC = 0.999
NORMAL_AGREE = 0.999
# end to end (each side renders its own fused map): the maps agree except on the oracle's ties, where a
# voxel's presence can differ; a sample whose corners include such a voxel can change the crossing
DEPTH_AGREE = 0.999
# colour (0..255): FP32 trilinear colour of FP32 running averages against FP64, on 99.9 % of the
# pixels (a direction whose combination weight vanishes at the evaluation point changes the mix)
COLOUR_TOL = 0.5
# a fusion weight is Lipschitz in the pixel normal (w_dir has slope 1/(2 theta - pi/2) per radian)
# and FP32 normals differ from FP64 ones by ~1e-7 rad: an absolute allowance per voxel
W_ABS = 1e-5
# sdf (units of tau): FP32 cross-product normals carry ~1e-5 rad error at 2-pixel baselines,
# times |x - p| <= tau, accumulated over the running average
SDF_TOL = 2e-4
# photometric rows: the keyframe sampling position is a single-precision projection (~1e-4 px at
# f = 525), which moves the bilinear gradient by |grad^2 I| 1e-4 px; intensities and gradients
# themselves are correctly rounded (exact integer intensity sums)
PHOTO_H_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    dt.lib()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def fuse_both(scene, frames, dense, voxel=0.01, tau=0.04, max_blocks=1 << 16, color=True):
    kw = dict(voxel_size=voxel, truncation=tau, dense_dim=64 if dense else 0, color=color)
    gm = dt.Map(dt.params(max_blocks=max_blocks, **kw))
    om = oracle.OracleMap(oracle.Params(**kw))
    for i in frames:
        f = scene.frame(i)
        gm.integrate(cu(f.depth), cu(f.rgb) if color else None, scene.K, f.pose)
        om.integrate(f.depth, f.rgb if color else None, scene.K, f.pose)
    torch.cuda.synchronize()
    return gm, om


def render_gpu(gm, K, T, color=True):
    d = torch.zeros(K.height, K.width, device=DEV)
    n = torch.zeros(K.height, K.width, 4, device=DEV)
    c = torch.zeros(K.height, K.width, 4, device=DEV) if color else None
    gm.render(K, T, d, n, c)
    torch.cuda.synchronize()
    return d.cpu().numpy(), n.cpu().numpy(), None if c is None else c.cpu().numpy()


def oracle_map_on_device(om, **kw):
    """The oracle's FP64 map, rounded to FP32, loaded into a device map (dtsdf_map_import)."""
    ob = om.bricks()
    vox = np.stack([om.brick(*b[:4]) for b in ob]).astype(np.float32)
    gm = dt.Map(dt.params(max_blocks=max(len(ob), 64), **kw))
    gm.import_bricks(ob[:, :4], vox)
    return gm


def compare_maps(gm, om):
    r = _compare(gm, om, sdf_tol=SDF_TOL, w_abs=W_ABS)
    print(f"map parity: {r['checked']} voxels checked in {r['bricks']} bricks; differing on ties: "
          f"{r['tie_keys']} keys, {r['tie_voxels']} voxels, {r['tie_colour']} colours")
    return r["checked"]


def test_exp_map_matches_matrix_exponential():
    rng = np.random.default_rng(7)
    for scale in (0.0, 1e-9, 1e-6, 1e-4, 1e-3, 1e-2, 0.3, 2.0):
        for dim in (6, 7):
            for _ in range(5):
                xi = rng.normal(size=dim) * scale
                assert np.allclose(dt.exp(xi), oicp.exp(xi), rtol=0, atol=2e-14 * max(1.0, scale * 10))


def test_dense_fusion_matches_oracle():
    s = scenes.tiny_scene(1)
    gm, om = fuse_both(s, range(10), dense=True)
    assert compare_maps(gm, om) > 50000


def test_hash_allocation_and_fusion_match_oracle():
    s = scenes.tiny_scene(1)
    gm, om = fuse_both(s, range(0, 10, 2), dense=False)
    st = gm.stats()
    assert st.error_flags == 0 and st.bricks == om.num_bricks()
    assert compare_maps(gm, om) > 20000


def test_hash_allocation_kinect_frames_match_up_to_ties():
    s = scenes.kinect_room(1)
    gm, om = fuse_both(s, range(0, 300, 60), dense=False, voxel=0.005, tau=0.02, max_blocks=1 << 18)
    coords, _ = gm.export()
    g, o = {tuple(c) for c in coords}, {tuple(b[:4]) for b in om.bricks()}
    diff = g ^ o
    print(f"kinect allocation: {len(o)} keys, {len(diff)} differ (all ties)")
    assert all(om.alloc_tie(*k) >= 0 for k in diff)
    assert len(diff) <= 1e-3 * len(o)


def _render_parity(gm, om, K, T, color=True):
    dg, ng, cg = render_gpu(gm, K, T, color)
    do, no, co, cok = om.render(K, T)
    hg, ho = dg > 0, do > 0
    agree = float(np.mean(hg == ho))
    both = hg & ho
    derr = np.abs(dg[both] - do[both])
    nerr = angles.between(ng[both][:, :3], no[both])
    cerr = None
    if color:
        cb = both & (cg[..., 3] > 0) & (cok > 0)
        cerr = np.abs(cg[cb][:, :3] - co[cb]).max(-1) if cb.any() else np.zeros(1)
    return agree, derr, nerr, cerr, both.sum()


def _report(tag, agree, derr, nerr, cerr):
    print(f"{tag}: mask {agree:.5f} depth max {derr.max():.2e} q999 {np.quantile(derr, 0.999):.2e} "
          f"normals <= 1e-3: {np.mean(nerr <= NORMAL_TOL):.5f} max {nerr.max():.2e} "
          f"colour q999 {np.quantile(cerr, 0.999):.3f} max {cerr.max():.3f}")


@pytest.mark.parametrize("fi", [0, 3, 5, 9])
def test_renderer_matches_oracle_on_the_same_map(fi):
    s = scenes.tiny_scene(1)
    om = oracle.OracleMap(oracle.Params(voxel_size=0.01, truncation=0.04, dense_dim=64))
    for i in range(10):
        f = s.frame(i)
        om.integrate(f.depth, f.rgb, s.K, f.pose)
    gm = oracle_map_on_device(om, voxel_size=0.01, truncation=0.04, dense_dim=64)
    T = s.poses[fi] @ scenes.perturbation(np.random.default_rng(fi), 1.0, 0.005)
    agree, derr, nerr, cerr, n = _render_parity(gm, om, s.K, T)
    _report(f"renderer pose {fi}", agree, derr, nerr, cerr)
    assert n > 5000
    assert agree >= MASK_AGREE, agree
    assert derr.max() <= DEPTH_TOL, derr.max()
    assert np.mean(nerr <= NORMAL_TOL) >= NORMAL_AGREE, np.mean(nerr <= NORMAL_TOL)
    assert np.quantile(cerr, 0.999) <= COLOUR_TOL


@pytest.mark.parametrize("fi", [0, 3, 5, 9])
def test_fuse_and_render_match_oracle_dense(fi):
    s = scenes.tiny_scene(1)
    gm, om = fuse_both(s, range(10), dense=True)
    T = s.poses[fi] @ scenes.perturbation(np.random.default_rng(fi), 1.0, 0.005)
    agree, derr, nerr, cerr, n = _render_parity(gm, om, s.K, T)
    _report(f"end to end pose {fi}", agree, derr, nerr, cerr)
    assert n > 5000
    assert agree >= MASK_AGREE, agree
    assert np.mean(derr <= DEPTH_TOL) >= DEPTH_AGREE, np.mean(derr <= DEPTH_TOL)
    assert np.mean(nerr <= NORMAL_TOL) >= NORMAL_AGREE, np.mean(nerr <= NORMAL_TOL)
    assert np.quantile(cerr, 0.999) <= COLOUR_TOL


def test_render_matches_oracle_hash_planes():
    s = scenes.planes_scene()
    s.noise_s0 = 0.001
    poses = [s.poses[0] @ scenes.perturbation(np.random.default_rng(k), 6.0, 0.1) for k in range(6)]
    s.poses = poses
    gm, om = fuse_both(s, range(6), dense=False, voxel=0.01, tau=0.04)
    T = poses[2] @ scenes.perturbation(np.random.default_rng(99), 2.0, 0.02)
    agree, derr, nerr, cerr, n = _render_parity(gm, om, s.K, T)
    _report("planes end to end", agree, derr, nerr, cerr)
    assert n > 5000 and agree >= MASK_AGREE and np.mean(derr <= DEPTH_TOL) >= DEPTH_AGREE
    assert np.mean(nerr <= NORMAL_TOL) >= NORMAL_AGREE
    # and the renderer alone, on the oracle's map
    gm2 = oracle_map_on_device(om, voxel_size=0.01, truncation=0.04)
    agree, derr, nerr, cerr, n = _render_parity(gm2, om, s.K, T)
    _report("planes renderer", agree, derr, nerr, cerr)
    assert n > 5000 and agree >= MASK_AGREE and derr.max() <= DEPTH_TOL and np.mean(nerr <= NORMAL_TOL) >= NORMAL_AGREE


def test_render_is_deterministic():
    s = scenes.tiny_scene(1)
    gm, _ = fuse_both(s, range(10), dense=True)
    a = render_gpu(gm, s.K, s.poses[4])
    b = render_gpu(gm, s.K, s.poses[4])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# --------------------------------------------------------------------- ICP --

def _analytic_ref(scene, T_ref, K):
    ref = scene.render(T_ref, K=K, noise=False, exact=True)
    n4 = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    n4[..., :3] = ref.normals
    n4[..., 3] = ref.depth
    n4[ref.depth == 0] = 0
    return ref.depth, n4


@pytest.mark.parametrize("sim3", [False, True])
@pytest.mark.parametrize("level", [0, 1, 2])
def test_icp_normal_equations_match_oracle(sim3, level):
    s = scenes.planes_scene()
    K = s.K
    T_ref = s.poses[0]
    rng = np.random.default_rng(3 + level)
    T_cur = T_ref @ scenes.perturbation(rng, 2.0, 0.02)
    cur = s.render(T_cur, noise=True)
    rd, rn = _analytic_ref(s, T_ref, K)
    dT = np.linalg.inv(T_ref) @ T_cur @ oicp.exp(rng.normal(size=6) * 0.01)
    if sim3:
        dT[:3, :3] *= 1.01
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_frame(cu(cur.depth), None, K, 0.1, 6.0, 0.02)
    opts = dt.icp_opts(levels=3, eps=(0.05, 0.1, 0.1), min_rows=1)
    T1, st = ic.step(cu(rd), cu(rn), K, level, dT, opts, sim3=sim3)
    # oracle on the same inputs
    pre = oracle.preprocess(cur.depth, K, 0.1, 6.0, 0.02)
    lv = oicp.pyramid(pre["z"], K, 3)[level]
    rows = oicp.geometric_rows(lv, rd, rn, K, dT, opts.eps[level], 0.1, sim3)
    H, g, E, n = oicp.normal_equations([rows])
    nt, tH, tg, tE = oicp.tie_bounds([rows])
    print(f"level {level} sim3 {sim3}: rows {st.rows} vs {n}, tie pixels {nt}")
    assert abs(st.rows - n) <= nt
    Hg = st.H_matrix()
    assert np.linalg.norm(Hg - H) <= 1e-5 * np.linalg.norm(H) + tH
    scale_g = np.abs(rows.J).T @ (rows.w * np.abs(rows.r)) + np.abs(rows.J).T @ rows.w * 1e-7
    assert np.all(np.abs(st.g_vector() - g) <= 1e-5 * np.abs(g) + 1e-3 * scale_g + tg)
    xi, ok = oicp.solve(H, g)
    assert ok and st.status == 0
    assert np.allclose(T1, oicp.exp(xi) @ dT, atol=1e-6)


@pytest.mark.parametrize("mode", ["f2kf", "f2f"])
def test_icp_photometric_rows_match_oracle(mode):
    """Photometric rows against a keyframe (f2kf) and against the previous frame, whose camera is
    the render camera (f2f: T_rs = I, Sec. 5)."""
    s = scenes.planes_scene()
    K = s.K
    T_ref = s.poses[0]
    rng = np.random.default_rng(21)
    T_kf = T_ref @ scenes.perturbation(rng, 3.0, 0.03)
    if mode == "f2f":
        T_kf = T_ref
    T_cur = T_ref @ scenes.perturbation(rng, 1.5, 0.015)
    cur = s.render(T_cur, noise=False)
    kf = s.render(T_kf, noise=False)
    rd, rn = _analytic_ref(s, T_ref, K)
    T_rs = np.eye(4) if mode == "f2f" else np.linalg.inv(T_kf) @ T_ref
    dT = np.linalg.inv(T_ref) @ T_cur
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_frame(cu(cur.depth), cu(cur.rgb), K, 0.1, 6.0, 0.02)
    ic.set_keyframe(cu(kf.rgb), K)
    opts = dt.icp_opts(levels=3, eps=(0.05, 0.1, 0.1), photo_thr=(0.3, 0.3, 0.3), lam=0.1, min_rows=1)
    for level in (0, 1):
        T1, st = ic.step(cu(rd), cu(rn), K, level, dT, opts, T_rs=T_rs)
        pre = oracle.preprocess(cur.depth, K, 0.1, 6.0, 0.02)
        lv = oicp.pyramid(pre["z"], K, 3, cur.rgb)[level]
        kI = oicp.pyramid(pre["z"], K, 3, kf.rgb)[level].I
        geo = oicp.geometric_rows(lv, rd, rn, K, dT, opts.eps[level], 0.1, False)
        ph = oicp.photometric_rows(lv, kI, K.scaled(level), T_rs, dT, opts.photo_thr[level], 0.1, 0.1, False)
        H, g, E, n = oicp.normal_equations([geo, ph])
        nt, tH, tg, tE = oicp.tie_bounds([geo, ph])
        rel = np.linalg.norm(st.H_matrix() - H) / np.linalg.norm(H)
        Hp = ph.J.T @ (ph.w[:, None] * ph.J)
        print(f"{mode} level {level}: photometric rows {st.rows_photo} vs {ph.J.shape[0]} (ties {ph.n_tie}), "
              f"geometric {st.rows - st.rows_photo} vs {geo.J.shape[0]} (ties {geo.n_tie}); H rel {rel:.2e}, "
              f"photometric share of |H| {np.linalg.norm(Hp) / np.linalg.norm(H):.2e}, tie bound {tH:.2e}")
        assert abs(st.rows_photo - ph.J.shape[0]) <= ph.n_tie
        assert abs((st.rows - st.rows_photo) - geo.J.shape[0]) <= geo.n_tie
        assert np.linalg.norm(st.H_matrix() - H) <= PHOTO_H_TOL * np.linalg.norm(H) + tH


@pytest.mark.parametrize("sim3", [False, True])
def test_icp_schedule_recovers_pose_like_oracle(sim3):
    s = scenes.planes_scene()
    K = s.K
    T_ref = s.poses[0]
    rng = np.random.default_rng(5)
    T_cur = T_ref @ scenes.perturbation(rng, 2.0, 0.02)
    scale = 1.04 if sim3 else 1.0
    cur = s.render(T_cur, noise=True, depth_scale=scale)
    rd, rn = _analytic_ref(s, T_ref, K)
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_frame(cu(cur.depth), None, K, 0.1, 6.0, 0.02)
    opts = dt.icp_opts(levels=3, iters=(10, 5, 4), eps=(0.02, 0.2, 0.3))
    Tdev = torch.eye(4, dtype=torch.float64, device=DEV)
    ic.solve(cu(rd), cu(rn), K, Tdev, opts, sim3=sim3)
    Tg = Tdev.cpu().numpy()
    pre = oracle.preprocess(cur.depth, K, 0.1, 6.0, 0.02)
    levels = oicp.pyramid(pre["z"], K, 3)
    st = oicp.Settings(sim3=sim3, eps=(0.02, 0.2, 0.3), iters=(10, 5, 4))
    To, _ = oicp.track(levels, rd, rn, K, np.eye(4), st)
    sg, so = np.cbrt(np.linalg.det(Tg[:3, :3])), np.cbrt(np.linalg.det(To[:3, :3]))
    assert abs(sg / so - 1) <= 1e-5
    Rg, Ro = Tg[:3, :3] / sg, To[:3, :3] / so
    ang = np.arccos(np.clip((np.trace(Rg.T @ Ro) - 1) / 2, -1, 1))
    assert ang <= 1e-4 and np.linalg.norm(Tg[:3, 3] - To[:3, 3]) <= 1e-4
    # and both recover the true motion to the noise level
    true = np.linalg.inv(T_ref) @ T_cur
    assert np.linalg.norm(To[:3, 3] - true[:3, 3]) < 5e-3


@pytest.mark.parametrize("sim3", [False, True])
def test_icp_lm_schedule_matches_oracle(sim3):
    """Levenberg-Marquardt (opts.lm = 1) against the oracle's LM schedule on a noisy frame whose
    gain ratios stay far from 0 (accept / reject decisions are not near a tie): same pose
    (1e-4 rad / 1e-4 m / 1e-5 relative scale), same number of evaluations, same rejections."""
    s = scenes.planes_scene()
    K = s.K
    T_ref = s.poses[0]
    rng = np.random.default_rng(5)
    T_cur = T_ref @ scenes.perturbation(rng, 2.0, 0.02)
    cur = s.render(T_cur, noise=True, depth_scale=1.04 if sim3 else 1.0)
    rd, rn = _analytic_ref(s, T_ref, K)
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_frame(cu(cur.depth), None, K, 0.1, 6.0, 0.02)
    opts = dt.icp_opts(levels=3, iters=(10, 5, 4), eps=(0.02, 0.2, 0.3), lm=True)
    Tdev = torch.eye(4, dtype=torch.float64, device=DEV)
    stats = torch.zeros(dt.STATS_BYTES, dtype=torch.uint8, device=DEV)
    ic.solve(cu(rd), cu(rn), K, Tdev, opts, sim3=sim3, stats_dev=stats)
    Tg = Tdev.cpu().numpy()
    st = dt.stats_from_device(stats)
    pre = oracle.preprocess(cur.depth, K, 0.1, 6.0, 0.02)
    levels = oicp.pyramid(pre["z"], K, 3)
    so_ = oicp.Settings(sim3=sim3, eps=(0.02, 0.2, 0.3), iters=(10, 5, 4), lm=True)
    To, log = oicp.track(levels, rd, rn, K, np.eye(4), so_)
    evals = [e for e in log if "mu" in e]
    assert any(not e["accepted"] for e in evals)
    assert all(e["rho"] is None or abs(e["rho"]) > 0.1 for e in evals)
    assert st.status == 0 and st.iterations == len(evals)
    sg, so = np.cbrt(np.linalg.det(Tg[:3, :3])), np.cbrt(np.linalg.det(To[:3, :3]))
    assert abs(sg / so - 1) <= 1e-5
    Rg, Ro = Tg[:3, :3] / sg, To[:3, :3] / so
    ang = np.arccos(np.clip((np.trace(Rg.T @ Ro) - 1) / 2, -1, 1))
    assert ang <= 1e-4 and np.linalg.norm(Tg[:3, 3] - To[:3, 3]) <= 1e-4


def test_icp_reduction_is_bitwise_deterministic():
    s = scenes.planes_scene()
    K = s.K
    cur = s.render(s.poses[0] @ scenes.perturbation(np.random.default_rng(1), 2, 0.02), noise=True)
    rd, rn = _analytic_ref(s, s.poses[0], K)
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_frame(cu(cur.depth), None, K, 0.1, 6.0, 0.02)
    opts = dt.icp_opts(levels=3, eps=(0.05, 0.1, 0.1))
    outs = [ic.step(cu(rd), cu(rn), K, 0, np.eye(4), opts) for _ in range(3)]
    for T, st in outs[1:]:
        assert np.array_equal(T, outs[0][0])
        assert bytes(st) == bytes(outs[0][1])


def test_degenerate_plane_reported():
    s = scenes.plane_scene()
    ref = s.render(s.poses[0], noise=False, exact=True)
    n4 = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    n4[..., :3] = ref.normals
    n4[..., 3] = ref.depth
    ic = dt.Icp(s.K.width, s.K.height, 1)
    ic.set_frame(cu(ref.depth), None, s.K, 0.1, 6.0, 0.02)
    T, st = ic.step(cu(ref.depth), cu(n4), s.K, 0, np.eye(4), dt.icp_opts(levels=1, eps=(0.05,)), sim3=True)
    assert st.status == dt.ERR_DEGENERATE and np.array_equal(T, np.eye(4))


def test_map_full_is_reported():
    s = scenes.tiny_scene(1)
    gm = dt.Map(dt.params(voxel_size=0.01, truncation=0.04, max_blocks=64))
    f = s.frame(0)
    gm.integrate(cu(f.depth), cu(f.rgb), s.K, f.pose)
    st = gm.stats()
    assert st.error_flags & 1 and st.bricks == 64
    with pytest.raises(dt.DtsdfError) as e:
        gm.integrate(cu(f.depth), cu(f.rgb), s.K, f.pose)
    assert e.value.status == dt.ERR_MAP_FULL


# ------------------------------------------------------------ precision form --

def _fuse_fp16(scene, frames, dense=True):
    kw = dict(voxel_size=0.01, truncation=0.04, dense_dim=64 if dense else 0, color=True)
    gm = dt.Map(dt.params(max_blocks=1 << 16, storage=dt.STORE_FP16, **kw))
    om = oracle.OracleMap(oracle.Params(**kw))
    for i in frames:
        f = scene.frame(i)
        gm.integrate(cu(f.depth), cu(f.rgb), scene.K, f.pose)
        om.integrate(f.depth, f.rgb, scene.K, f.pose)
    torch.cuda.synchronize()
    return gm, om


def test_fp16_storage_map_matches_oracle():
    """FP16 sdf, half weight in a u16, u8 colour: same allocation and presence as the oracle,
    values within the storage quantisation accumulated over the running averages."""
    s = scenes.tiny_scene(1)
    gm, om = _fuse_fp16(s, range(10))
    coords, vox = gm.export()
    idx = {tuple(c): i for i, c in enumerate(coords)}
    n = 0
    errs = []
    for b in om.bricks():
        g = vox[idx[tuple(b[:4])]].astype(np.float64)
        o = om.brick(*b[:4])
        tie = (om.brick_ties(*b[:4]) & 1) > 0
        assert np.all(((g[:, 1] > 0) == (o[:, 1] > 0)) | tie)
        p = (o[:, 1] > 0) & (g[:, 1] > 0) & ~tie
        if p.any():
            errs.append(np.abs(g[p, 0] - o[p, 0]))
            assert np.all(np.abs(g[p, 1] - o[p, 1]) <= 0.01 * o[p, 1] + 1e-5)
            n += p.sum()
    assert n > 50000
    # half precision: 2^-11 relative per stored sdf and weight, re-rounded at every update and
    # carried through the running averages
    e = np.concatenate(errs)
    assert np.quantile(e, 0.999) <= 2e-3 and e.max() <= 0.05, (np.quantile(e, 0.999), e.max())


@pytest.mark.parametrize("fi", [0, 5])
def test_fp16_render_matches_oracle(fi):
    s = scenes.tiny_scene(1)
    gm, om = _fuse_fp16(s, range(10))
    T = s.poses[fi] @ scenes.perturbation(np.random.default_rng(fi), 1.0, 0.005)
    dg, ng, cg = render_gpu(gm, s.K, T, True)
    do, no, co, cok = om.render(s.K, T)
    hg, ho = dg > 0, do > 0
    agree = float(np.mean(hg == ho))
    both = hg & ho
    assert both.sum() > 5000
    derr = np.abs(dg - do)
    # The FP16 field differs from the FP64 one by the storage rounding, so a sign test at a
    # sample whose stored value is within that rounding of zero can go the other way: the ray
    # then stops at a neighbouring crossing. Those pixels are counted, not excluded.
    close = both & (derr <= DEPTH_TOL)
    frac = close.sum() / both.sum()
    nerr = angles.between(ng[both][:, :3], no[both])
    cb = close & (cg[..., 3] > 0) & (cok > 0)
    cerr = np.abs(cg[cb][:, :3] - co[cb]).max(-1)
    print(f"fp16 fi={fi}: mask {agree:.5f} depth<=1e-4 {frac:.5f} median {np.median(derr[both]):.2e} "
          f"max {derr[both].max():.3e} normals {np.mean(nerr <= NORMAL_TOL):.4f} "
          f"colour q999 {np.quantile(cerr, 0.999):.2f} max {cerr.max():.2f}")
    assert agree >= MASK_AGREE, agree
    assert frac >= FP16_DEPTH_FRAC and np.median(derr[both]) <= 1e-5, (frac, np.median(derr[both]))
    assert np.mean(nerr <= NORMAL_TOL) >= 0.99, np.mean(nerr <= NORMAL_TOL)
    # u8 colour channels re-rounded at every update, mixed with a log-coded colour weight
    assert np.quantile(cerr, 0.999) <= 3.0, np.quantile(cerr, 0.999)


@pytest.mark.parametrize("sim3", [False, True])
def test_kahan_reduction_matches_oracle(sim3):
    s = scenes.planes_scene()
    K = s.K
    T_ref = s.poses[0]
    rng = np.random.default_rng(31)
    T_cur = T_ref @ scenes.perturbation(rng, 2.0, 0.02)
    cur = s.render(T_cur, noise=True)
    rd, rn = _analytic_ref(s, T_ref, K)
    dT = np.linalg.inv(T_ref) @ T_cur @ oicp.exp(rng.normal(size=6) * 0.01)
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_frame(cu(cur.depth), None, K, 0.1, 6.0, 0.02)
    opts = dt.icp_opts(levels=3, eps=(0.05, 0.1, 0.1), min_rows=1, kahan=True)
    T1, st = ic.step(cu(rd), cu(rn), K, 0, dT, opts, sim3=sim3)
    pre = oracle.preprocess(cur.depth, K, 0.1, 6.0, 0.02)
    lv = oicp.pyramid(pre["z"], K, 3)[0]
    rows = oicp.geometric_rows(lv, rd, rn, K, dT, 0.05, 0.1, sim3)
    H, g, E, nr = oicp.normal_equations([rows])
    assert st.rows == nr
    assert np.linalg.norm(st.H_matrix() - H) <= 1e-5 * np.linalg.norm(H)
    xi, ok = oicp.solve(H, g)
    assert np.allclose(T1, oicp.exp(xi) @ dT, atol=1e-6)
