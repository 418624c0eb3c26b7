"""Voxel recycling (Sec. 3; dtsdf_recycle) against the oracle's: the same bricks leave the map,
the freed bricks are handed out again before the pool grows, and fusion and rendering after
recycling match the oracle.

Tolerances: a brick's removal is decided by comparing its weighted voxels with the threshold, in
FP32 on the device and FP64 in the oracle, so bricks whose smallest weighted sdf lies within 1e-3
of the threshold may go either way and are excluded from the set and value comparisons (none
occur in practice); voxel values as the fusion parity (sdf within 2e-4, weights within
1e-4 w + 1e-5); renders as the direct render parity (mask >= 99.9 %, depth within 1e-4 m)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import scenes
import paper_2301_12796_gb300 as dt
from paper_2301_12796_gb300 import build as B

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
THR = 0.75


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    dt.lib()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _pool_count(gm):
    n = ctypes.c_int64()
    dt.check(dt.lib().dtsdf_map_export(gm._h, None, None, 0, ctypes.byref(n), None), "export")
    return int(n.value)


def _oracle_snapshot(om):
    return {tuple(b[:4]): om.brick(*b[:4]) for b in om.bricks()}


def _ties(snap):
    out = set()
    for k, v in snap.items():
        w = v[:, 1] > 0
        if w.any() and abs(float(v[w, 0].min()) - THR) < 1e-3:
            out.add(k)
    return out


def _fuse(gm, om, s, frames):
    for i in frames:
        f = s.frame(i)
        gm.integrate(cu(f.depth), cu(f.rgb), s.K, f.pose)
        om.integrate(f.depth, f.rgb, s.K, f.pose)
    torch.cuda.synchronize()


def test_recycle_and_reuse_match_oracle():
    s = scenes.tiny_scene(1)
    kw = dict(voxel_size=0.01, truncation=0.04)
    gm = dt.Map(dt.params(max_blocks=1 << 16, **kw))
    om = oracle.OracleMap(oracle.Params(**kw))
    _fuse(gm, om, s, range(6))
    ties = _ties(_oracle_snapshot(om))
    pool0 = _pool_count(gm)
    live0 = gm.stats().bricks
    n_g = gm.recycle(THR)
    n_o = om.recycle(THR)
    assert n_o > 20 and abs(n_g - n_o) <= len(ties)
    coords, vox = gm.export()
    gset = {tuple(c) for c in coords}
    oset = {tuple(b[:4]) for b in om.bricks()}
    assert all(k in ties or om.alloc_tie(*k) >= 0 for k in gset ^ oset)
    assert gm.stats().bricks == len(gset) == live0 - n_g
    assert gm.recycle(THR) == 0
    # fusion after recycling: removed bricks that are observed again come from the free ring
    _fuse(gm, om, s, range(6, 10))
    coords, vox = gm.export()
    gset = {tuple(c) for c in coords}
    oset = {tuple(b[:4]) for b in om.bricks()}
    assert all(k in ties or om.alloc_tie(*k) >= 0 for k in gset ^ oset)
    live1 = gm.stats().bricks
    assert live1 == len(gset)
    realloc = live1 - (live0 - n_g)
    assert _pool_count(gm) == pool0 + max(0, realloc - n_g)
    idx = {tuple(c): i for i, c in enumerate(coords)}
    checked = 0
    for b in om.bricks():
        k = tuple(b[:4])
        if k in ties or k not in idx or om.alloc_tie(*k) >= 0:
            continue
        g = vox[idx[k]].astype(np.float64)
        o = om.brick(*k)
        tie = (om.brick_ties(*k) & 1) > 0
        assert np.all(((g[:, 1] > 0) == (o[:, 1] > 0)) | tie)
        w = (o[:, 1] > 0) & (g[:, 1] > 0) & ~tie
        assert np.max(np.abs(g[w, 0] - o[w, 0]), initial=0.0) <= 2e-4
        assert np.all(np.abs(g[w, 1] - o[w, 1]) <= 1e-4 * o[w, 1] + 1e-5)
        checked += 1
    assert checked > 500
    # the render of the recycled and refused map
    T = s.poses[7] @ scenes.perturbation(np.random.default_rng(7), 1.0, 0.005)
    K = s.K
    d = torch.zeros(K.height, K.width, device=DEV)
    n = torch.zeros(K.height, K.width, 4, device=DEV)
    gm.render(K, T, d, n)
    torch.cuda.synchronize()
    d = d.cpu().numpy()
    do, no, _, _ = om.render(K, T)
    assert np.mean((d > 0) == (do > 0)) >= 0.999
    both = (d > 0) & (do > 0)
    assert np.max(np.abs(d[both] - do[both])) <= 1e-4


def test_recycle_rejects_dense_maps_and_bad_thresholds():
    gm = dt.Map(dt.params(max_blocks=1 << 12, voxel_size=0.01, truncation=0.04, dense_dim=64))
    with pytest.raises(dt.DtsdfError):
        gm.recycle(THR)
    gm = dt.Map(dt.params(max_blocks=1 << 12, voxel_size=0.01, truncation=0.04))
    for bad in (0.0, -1.0, 1.5):
        with pytest.raises(dt.DtsdfError):
            gm.recycle(bad)
    assert gm.recycle(THR) == 0
