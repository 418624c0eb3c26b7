"""The free-space combination render (Sec. 4, Alg. 1; dtsdf_render_freespace) against the
oracle's, on the oracle's own map loaded into the device (the renderer alone) and end to end.

Tolerances: the free / occupied decision of a sample, the transition tests and the taking-part
test (w_dir > 0) are floating-point comparisons taken in FP32 on the device and FP64 in the oracle,
so a ray whose decision sits at a tie can stop at a different crossing; the bar is the direct
render's one with a wider share: hit masks agree on >= 99.5 % of the pixels, depth within 1e-4 m
on >= 99.5 % and normals within 1e-3 rad on >= 99 % of the pixels both hit."""
import numpy as np
import pytest
import torch

import angles
import oracle
import scenes
import paper_2301_12796_gb300 as dt
from paper_2301_12796_gb300 import build as B

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    dt.lib()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _render(gm, K, T):
    d = torch.zeros(K.height, K.width, device=DEV)
    n = torch.zeros(K.height, K.width, 4, device=DEV)
    c = torch.full((K.height, K.width, 4), 7.0, device=DEV)
    gm.render_freespace(K, T, d, n, c)
    torch.cuda.synchronize()
    assert not c.any()  # no colour in this mode
    n = n.cpu().numpy()
    d = d.cpu().numpy()
    assert np.array_equal(n[..., 3], d)  # depth in w, as the direct render
    return d, n


def _compare(d, n, do, no):
    hg, ho = d > 0, do > 0
    agree = float(np.mean(hg == ho))
    both = hg & ho
    derr = np.abs(d[both] - do[both])
    nerr = angles.between(n[both][:, :3], no[both])
    return agree, derr, nerr, int(both.sum())


@pytest.mark.parametrize("fi", [1, 5, 8])
def test_freespace_render_matches_oracle_on_the_same_map(fi):
    s = scenes.tiny_scene(1)
    om = oracle.OracleMap(oracle.Params(voxel_size=0.01, truncation=0.04, dense_dim=64))
    for i in range(10):
        f = s.frame(i)
        om.integrate(f.depth, f.rgb, s.K, f.pose)
    ob = om.bricks()
    vox = np.stack([om.brick(*b[:4]) for b in ob]).astype(np.float32)
    gm = dt.Map(dt.params(max_blocks=max(len(ob), 64), voxel_size=0.01, truncation=0.04, dense_dim=64))
    gm.import_bricks(ob[:, :4], vox)
    T = s.poses[fi] @ scenes.perturbation(np.random.default_rng(fi), 1.0, 0.005)
    d, n = _render(gm, s.K, T)
    do, no = om.render_freespace(s.K, T)
    agree, derr, nerr, nb = _compare(d, n, do, no)
    assert nb > 5000
    assert agree >= 0.995, agree
    assert np.mean(derr <= 1e-4) >= 0.995, (np.mean(derr <= 1e-4), derr.max())
    assert np.mean(nerr <= 1e-3) >= 0.99, np.mean(nerr <= 1e-3)


def test_freespace_render_fused_on_both_sides_planes():
    """End to end on the planes scene (fused on each side from the same frames): the linear
    fields make both renders the analytic intersection where one direction takes part."""
    s = scenes.planes_scene()
    K = s.K
    kw = dict(voxel_size=0.01, truncation=0.04)
    gm = dt.Map(dt.params(max_blocks=1 << 16, color=False, **kw))
    om = oracle.OracleMap(oracle.Params(color=False, **kw))
    rng = np.random.default_rng(3)
    poses = [s.poses[0] @ scenes.perturbation(rng, 3.0, 0.03) for _ in range(4)]
    for i, T in enumerate(poses):
        f = s.render(T, frame_id=i, noise=False)
        gm.integrate(cu(f.depth), None, K, T)
        om.integrate(f.depth, None, K, T)
    T = s.poses[0] @ scenes.perturbation(rng, 1.0, 0.01)
    d, n = _render(gm, K, T)
    do, no = om.render_freespace(K, T)
    agree, derr, nerr, nb = _compare(d, n, do, no)
    assert nb > 0.8 * K.width * K.height
    assert agree >= 0.995 and np.mean(derr <= 1e-4) >= 0.995, (agree, np.mean(derr <= 1e-4))
    # and the direct render finds the same surfaces
    d0 = torch.zeros(K.height, K.width, device=DEV)
    n0 = torch.zeros(K.height, K.width, 4, device=DEV)
    gm.render(K, T, d0, n0)
    d0 = d0.cpu().numpy()
    both = (d0 > 0) & (d > 0)
    assert np.median(np.abs(d0[both] - d[both])) < 1e-4
