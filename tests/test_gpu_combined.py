"""Combined-TSDF render mode (dtsdf_render_combined) against the FP64 oracle's combination and
ray-cast, on the oracle's own map loaded into the device map: the tiny dense room at several
poses, the Kinect-shaped room at full size on sampled rays, and the conditional combination
(the stored field is reused after a small motion and recomputed after a large one).

Tolerances as for the direct render: hit mask >= 99.9 %, depth <= 1e-4 m and normals
<= 1e-3 rad on >= 99.9 % of the pixels both sides hit, colour <= 0.5 of 255."""
import numpy as np
import pytest

import angles
import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2301_12796_gb300 as dt  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def device_copy(om, **kw):
    ob = om.bricks()
    vox = np.stack([om.brick(*b[:4]) for b in ob]).astype(np.float32)
    gm = dt.Map(dt.params(max_blocks=len(ob) + 64, **kw))
    gm.import_bricks(ob[:, :4], vox)
    return gm


def render_comb(gm, K, T):
    d = torch.zeros(K.height, K.width, device=DEV)
    n = torch.zeros(K.height, K.width, 4, device=DEV)
    c = torch.zeros(K.height, K.width, 4, device=DEV)
    gm.render_combined(K, T, d, n, c)
    torch.cuda.synchronize()
    return d.cpu().numpy(), n.cpu().numpy(), c.cpu().numpy()


def compare(g, o, pix=None):
    dg, ng, cg = g
    do, no, co, cok = o
    if pix is not None:
        dg, ng, cg = dg[pix[:, 1], pix[:, 0]], ng[pix[:, 1], pix[:, 0]], cg[pix[:, 1], pix[:, 0]]
    hg, ho = dg > 0, do > 0
    both = hg & ho
    derr = np.abs(dg[both] - do[both])
    nerr = angles.between(ng[both][..., :3], no[both])
    cb = both & (cg[..., 3] > 0) & (cok > 0)
    cerr = np.abs(cg[cb][..., :3] - co[cb]).max() if cb.any() else 0.0
    return float(np.mean(hg == ho)), derr, nerr, cerr, int(both.sum())


@pytest.fixture(scope="module")
def tiny():
    s = scenes.tiny_scene(1)
    kw = dict(voxel_size=0.01, truncation=0.04, dense_dim=64, color=True)
    om = oracle.OracleMap(oracle.Params(**kw))
    for i in range(10):
        f = s.frame(i)
        om.integrate(f.depth, f.rgb, s.K, f.pose)
    return s, om, kw


@pytest.mark.parametrize("fi", [0, 4, 8])
def test_combined_render_matches_oracle(tiny, fi):
    s, om, kw = tiny
    gm = device_copy(om, **kw)
    T = s.poses[fi] @ scenes.perturbation(np.random.default_rng(fi), 1.0, 0.005)
    g = render_comb(gm, s.K, T)  # first call: boot-up, the whole frustum is combined at T
    om.combine(T[:3, 3])
    agree, derr, nerr, cerr, n = compare(g, om.render_combined(s.K, T))
    print(f"combined fi={fi}: mask {agree:.5f} depth max {derr.max():.2e} normals {np.mean(nerr <= 1e-3):.5f}")
    assert n > 5000
    assert agree >= 0.999
    assert np.mean(derr <= 1e-4) >= 0.999 and np.median(derr) < 1e-6
    assert np.mean(nerr <= 1e-3) >= 0.999
    assert cerr <= 0.5


def test_conditional_combination_reuses_and_recomputes(tiny):
    s, om, kw = tiny
    gm = device_copy(om, **kw)
    K = s.K
    T1 = s.poses[3]
    for _ in range(5):  # boot-up: five recombinations at T1
        render_comb(gm, K, T1)
    T2 = T1 @ scenes.perturbation(np.random.default_rng(2), 1.0, 0.01)  # small motion: field kept
    g2 = render_comb(gm, K, T2)
    om.combine(T1[:3, 3])
    agree, derr, nerr, _, _ = compare(g2, om.render_combined(K, T2))
    assert agree >= 0.999 and np.mean(derr <= 1e-4) >= 0.999 and np.mean(nerr <= 1e-3) >= 0.999
    T3 = s.poses[7]  # large motion: recombined at T3
    g3 = render_comb(gm, K, T3)
    om.combine(T3[:3, 3])
    agree, derr, nerr, _, _ = compare(g3, om.render_combined(K, T3))
    assert agree >= 0.999 and np.mean(derr <= 1e-4) >= 0.999 and np.mean(nerr <= 1e-3) >= 0.999
    # a reset forces the recombination at the next pose even for a small motion
    gm.combined_reset()
    T4 = T3 @ scenes.perturbation(np.random.default_rng(4), 0.5, 0.005)
    g4 = render_comb(gm, K, T4)
    om.combine(T4[:3, 3])
    agree, derr, _, _, _ = compare(g4, om.render_combined(K, T4))
    assert agree >= 0.999 and np.mean(derr <= 1e-4) >= 0.999


def test_combined_render_full_size_sampled():
    s = scenes.kinect_room(1)
    kw = dict(voxel_size=0.005, truncation=0.02, color=True, z_max=s.z_max)
    om = oracle.OracleMap(oracle.Params(**kw))
    for i in range(0, 300, 20):
        f = s.frame(i)
        om.integrate(f.depth, f.rgb, s.K, f.pose)
    gm = device_copy(om, **kw)
    K, T = s.K, s.poses[150]
    g = render_comb(gm, K, T)
    om.combine(T[:3, 3])
    vv, uu = np.mgrid[0:K.height:4, 0:K.width:4]
    pix = np.stack([uu.ravel(), vv.ravel()], 1).astype(np.int32)
    agree, derr, nerr, cerr, n = compare(g, om.render_combined(K, T, pix), pix)
    print(f"combined full size: mask {agree:.5f} depth<=1e-4 {np.mean(derr <= 1e-4):.5f} "
          f"normals {np.mean(nerr <= 1e-3):.5f} colour {cerr:.3f}")
    assert n > 10000 and agree >= 0.999
    assert np.mean(derr <= 1e-4) >= 0.999
    assert np.mean(nerr <= 1e-3) >= 0.999


def test_combined_render_after_recycling_matches_oracle():
    """Recycling detaches bricks, so the next combined render recombines its whole view: the
    oracle's hash map is loaded into the device, combined renders run past the boot-up phase,
    both sides recycle, and the next combined render is bit-identical to the combined render of
    a fresh device copy of the recycled oracle map and matches the oracle's combination. Blocks
    that lost a direction next to blocks that keep it test that every combined voxel is formed
    from its own block's directions."""
    s = scenes.tiny_scene(1)
    kw = dict(voxel_size=0.01, truncation=0.04, color=True)
    om = oracle.OracleMap(oracle.Params(**kw))
    for i in range(10):
        f = s.frame(i)
        om.integrate(f.depth, f.rgb, s.K, f.pose)
    gm = device_copy(om, **kw)
    T = s.poses[5] @ scenes.perturbation(np.random.default_rng(3), 1.0, 0.005)
    for _ in range(6):
        g0 = render_comb(gm, s.K, T)
    om.combine(T[:3, 3])
    agree, derr, nerr, cerr, n = compare(g0, om.render_combined(s.K, T))
    assert agree >= 0.999 and np.mean(derr <= 1e-4) >= 0.999 and np.mean(nerr <= 1e-3) >= 0.999
    n_g, n_o = gm.recycle(0.75), om.recycle(0.75)
    assert n_o > 20 and abs(n_g - n_o) <= 2  # a brick at the threshold may go either way
    g = render_comb(gm, s.K, T)
    fresh = render_comb(device_copy(om, **kw), s.K, T)
    if n_g == n_o:
        for a, b in zip(g, fresh):
            assert np.array_equal(a, b)
    om.combine(T[:3, 3])
    agree, derr, nerr, cerr, n = compare(g, om.render_combined(s.K, T))
    print(f"after recycling: mask {agree:.5f} depth {np.mean(derr <= 1e-4):.5f} normals {np.mean(nerr <= 1e-3):.5f}")
    assert n > 5000 and agree >= 0.999
    assert np.mean(derr <= 1e-4) >= 0.999
    assert np.mean(nerr <= 1e-3) >= 0.999


@pytest.mark.parametrize("dense", [True, False])
def test_fp16_combined_render_matches_oracle_on_the_same_values(dense):
    """FP16 storage form: the combine pass stages half-precision bricks (4-byte voxels, a brick
    starting 0, 4, 8 or 12 bytes past a 16-byte boundary). The map is fused on the device in FP16,
    and the oracle is given the map's own (decoded) voxel values, so both combine and ray-cast the
    same field and the FP32 bars apply. The hash map has blocks whose upper neighbours hold
    directions the block lacks."""
    s = scenes.tiny_scene(1)
    kw = dict(voxel_size=0.01, truncation=0.04, dense_dim=64 if dense else 0, color=True)
    gm = dt.Map(dt.params(max_blocks=1 << 16, storage=dt.STORE_FP16, **kw))
    for i in range(10):
        f = s.frame(i)
        gm.integrate(torch.from_numpy(f.depth).to(DEV), torch.from_numpy(np.ascontiguousarray(f.rgb)).to(DEV),
                     s.K, f.pose)
    torch.cuda.synchronize()
    coords, vox = gm.export()
    om = oracle.OracleMap(oracle.Params(**kw))
    for c, v in zip(coords, vox):
        om.set_brick(int(c[0]), int(c[1]), int(c[2]), int(c[3]), v.astype(np.float64))
    for fi in (2, 6):
        T = s.poses[fi] @ scenes.perturbation(np.random.default_rng(fi), 1.0, 0.005)
        gm.combined_reset()
        g = render_comb(gm, s.K, T)
        om.combine(T[:3, 3])
        agree, derr, nerr, cerr, n = compare(g, om.render_combined(s.K, T))
        print(f"fp16 combined dense={dense} fi={fi}: mask {agree:.5f} depth max {derr.max():.2e} "
              f"normals {np.mean(nerr <= 1e-3):.5f} colour {cerr:.3f}")
        assert n > 5000
        assert agree >= 0.999
        assert np.mean(derr <= 1e-4) >= 0.999 and np.median(derr) < 1e-6
        assert np.mean(nerr <= 1e-3) >= 0.999
        assert cerr <= 0.5


def test_incremental_combination_takes_new_blocks_and_their_neighbours():
    """Conditional combination with new blocks (Sec. 4): after the boot-up the stored field is
    reused, and only blocks that received bricks since the last combination are combined, with the
    26 blocks around each of them, whose stored voxels next to a new block (the layer at local 8
    a block keeps for its upper neighbours, the gradient stencils reaching into the new block)
    depend on its bricks. The oracle's hash map is loaded without a slab of blocks, combined at
    T through the boot-up, then given the slab (nothing else changes): the next combined render at
    T recombines incrementally and must match the oracle's combination of the whole map at T."""
    s = scenes.tiny_scene(1)
    kw = dict(voxel_size=0.01, truncation=0.04, color=True)
    om = oracle.OracleMap(oracle.Params(**kw))
    for i in range(10):
        f = s.frame(i)
        om.integrate(f.depth, f.rgb, s.K, f.pose)
    ob = om.bricks()
    vox = np.stack([om.brick(*b[:4]) for b in ob]).astype(np.float32)
    slab = ob[:, 0] == int(np.median(ob[:, 0]))
    assert 100 < slab.sum() < len(ob) - 100
    gm = dt.Map(dt.params(max_blocks=len(ob) + 64, **kw))
    gm.import_bricks(ob[~slab, :4], vox[~slab])
    T = s.poses[5]
    for _ in range(5):  # boot-up: the whole frustum is combined at T
        render_comb(gm, s.K, T)
    gm.import_bricks(ob[slab, :4], vox[slab])
    blocks_before, _ = gm.combined_blocks()
    g = render_comb(gm, s.K, T)  # sixth call, same pose: incremental
    om.combine(T[:3, 3])
    agree, derr, nerr, cerr, n = compare(g, om.render_combined(s.K, T))
    print(f"incremental: mask {agree:.5f} depth<=1e-4 {np.mean(derr <= 1e-4):.5f} normals {np.mean(nerr <= 1e-3):.5f} "
          f"colour {cerr:.3f}, blocks {blocks_before} -> {gm.combined_blocks()[0]}")
    assert n > 5000
    assert agree >= 0.999
    assert np.mean(derr <= 1e-4) >= 0.999 and np.median(derr) < 1e-6
    assert np.mean(nerr <= 1e-3) >= 0.999
    assert cerr <= 0.5


def test_fp16_combined_render_full_size_sampled():
    """The FP16 combine pass at the benchmark's scale: the Kinect-shaped room fused on the device
    in FP16 from 15 of its frames (tens of thousands of staged bricks, starting at every 4-byte
    offset from a 16-byte boundary), the oracle given the map's decoded values, both combined at
    a trajectory pose and compared on every fourth pixel at the FP32 bars."""
    s = scenes.kinect_room(1)
    kw = dict(voxel_size=0.005, truncation=0.02, color=True, z_max=s.z_max)
    gm = dt.Map(dt.params(max_blocks=1 << 18, storage=dt.STORE_FP16, **kw))
    for i in range(0, 300, 20):
        f = s.frame(i)
        gm.integrate(torch.from_numpy(f.depth).to(DEV), torch.from_numpy(np.ascontiguousarray(f.rgb)).to(DEV),
                     s.K, f.pose)
    torch.cuda.synchronize()
    coords, vox = gm.export()
    assert len(coords) > 20000
    om = oracle.OracleMap(oracle.Params(**kw))
    for c, v in zip(coords, vox):
        om.set_brick(int(c[0]), int(c[1]), int(c[2]), int(c[3]), v.astype(np.float64))
    K, T = s.K, s.poses[150]
    g = render_comb(gm, K, T)
    om.combine(T[:3, 3])
    vv, uu = np.mgrid[0:K.height:4, 0:K.width:4]
    pix = np.stack([uu.ravel(), vv.ravel()], 1).astype(np.int32)
    agree, derr, nerr, cerr, n = compare(g, om.render_combined(K, T, pix), pix)
    print(f"fp16 combined full size: {len(coords)} bricks, mask {agree:.5f} depth<=1e-4 {np.mean(derr <= 1e-4):.5f} "
          f"normals {np.mean(nerr <= 1e-3):.5f} colour {cerr:.3f}")
    assert n > 10000 and agree >= 0.999
    assert np.mean(derr <= 1e-4) >= 0.999
    assert np.mean(nerr <= 1e-3) >= 0.999
    assert cerr <= 0.5
