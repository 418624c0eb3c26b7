"""Input preprocessing, bilateral filters and the post-fusion error through the C ABI
(dtsdf_preprocess, dtsdf_set_filters, dtsdf_icp_set_filters, dtsdf_depth_mae) against the oracle.

Tolerances: unfiltered preprocessing: the kept and normal masks are identical (the filter compares
differences of input depths, exact in either precision near its threshold), points within 1e-7
relative and normals within 1e-6 rad (both formed in double precision and rounded once), except
at the oracle's orientation ties, where the normal may point the other way; filtered depth within 1e-5 relative (FP32 sums of up to 121 weighted
taps against FP64) with identical presence masks; filtered normals within 1e-3 rad on 99.9 % of
the pixels with a normal (a normal whose camera-facing decision flips at a grazing pixel differs
by pi); the MAE sums within 1e-12 relative (FP64 on both sides, different summation order) and
the counts exact."""
import numpy as np
import pytest
import torch

import angles
import oracle
from oracle import filters as OF
import scenes
import paper_2301_12796_gb300 as dt
from paper_2301_12796_gb300 import build as B

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
ZMIN, ZMAX, DSUP = 0.1, 6.0, 0.02


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    dt.lib()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _frames():
    s = scenes.tiny_scene(1)
    return s, [s.frame(i) for i in range(10)]


def _angles(a, b):
    return angles.between(a, b)


def test_unfiltered_preprocessing_matches_oracle():
    s, frames = _frames()
    for f in frames[:3]:
        P, N = dt.preprocess(cu(f.depth), s.K, ZMIN, ZMAX, DSUP)
        torch.cuda.synchronize()
        P, N = P.cpu().numpy(), N.cpu().numpy()
        o = oracle.preprocess(f.depth, s.K, ZMIN, ZMAX, DSUP)
        assert np.array_equal(P[..., 3] > 0, o["ok"] > 0)
        assert np.array_equal(N[..., 3] > 0, o["nok"] > 0)
        ok = o["ok"] > 0
        assert np.all(np.abs(P[ok][:, :3] - o["P"][ok]) <= 1e-7 * np.linalg.norm(o["P"][ok], axis=-1)[:, None])
        nk = o["nok"] > 0
        ang = _angles(N[nk][:, :3].astype(np.float64), o["n"][nk])
        tie = o["tie"][nk] > 0
        print(f"normals: max {ang[~tie].max():.2e} rad off ties, {tie.sum()} orientation ties")
        assert np.all((ang <= 1e-6) | (tie & (ang >= np.pi - 1e-6)))


@pytest.mark.parametrize("which", ["depth", "normals", "both"])
def test_bilateral_filters_match_oracle(which):
    s, frames = _frames()
    f = dt.filter_opts(depth=which != "normals", normals=which != "depth")
    for fr in frames[:3]:
        P, N = dt.preprocess(cu(fr.depth), s.K, ZMIN, ZMAX, DSUP, f)
        torch.cuda.synchronize()
        P, N = P.cpu().numpy(), N.cpu().numpy()
        z = oracle.preprocess(fr.depth, s.K, ZMIN, ZMAX, DSUP)["z"].astype(np.float64)
        if f.depth_radius:
            z = OF.bilateral_depth(z, 5, 5.0, 0.025)
        valid = z > 0
        assert np.array_equal(P[..., 3] > 0, valid)
        np.testing.assert_allclose(P[..., 2][valid], z[valid], rtol=1e-5)
        n, has = OF.normals(OF.backproject(z, s.K), valid)
        if f.normal_radius:
            n = OF.bilateral_normals(n, has, 5, 2.5, 5.0)
        assert np.array_equal(N[..., 3] > 0, has)
        ang = _angles(N[..., :3][has].astype(np.float64), n[has])
        assert np.mean(ang <= 1e-3) >= 0.999, (which, np.mean(ang <= 1e-3), np.max(ang))


def test_filters_in_fusion_and_icp():
    """A map and an ICP context with both filters: the post-fusion error (Sec. 8.2) of the map
    fused with the filtered preprocessing stays at the level of the unfiltered one (most pixels
    within 3 mm; the mean is dominated by silhouette pixels that hit another surface) and equals
    the mean computed on the host from the same images; ICP converges on the filtered pyramid."""
    s, frames = _frames()
    K = s.K
    f = dt.filter_opts()
    maes, medians = {}, {}
    for name, filt in (("off", None), ("on", f)):
        gm = dt.Map(dt.params(max_blocks=1 << 16, voxel_size=0.01, truncation=0.04, color=False))
        gm.set_filters(filt)
        for fr in frames:
            gm.integrate(cu(fr.depth), None, K, fr.pose)
        d = torch.zeros(K.height, K.width, device=DEV)
        n = torch.zeros(K.height, K.width, 4, device=DEV)
        tot = np.zeros(2)
        errs = []
        for fr in frames:
            gm.render(K, fr.pose, d, n)
            out = dt.depth_mae(d, cu(fr.depth))
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            ref = OF.depth_mae(d.cpu().numpy(), fr.depth)
            assert int(got[1]) == ref[1] and got[0] == pytest.approx(ref[0], rel=1e-12)
            tot += got
            dd = d.cpu().numpy()
            both = (dd > 0) & (fr.depth > 0)
            errs.append(np.abs(dd - fr.depth)[both])
        maes[name] = tot[0] / tot[1]
        medians[name] = float(np.median(np.concatenate(errs)))
    assert medians["off"] < 3e-3 and medians["on"] < 3e-3, (medians, maes)
    assert maes["on"] < 1.25 * maes["off"], maes
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_filters(f)
    rd, rn = torch.zeros(K.height, K.width, device=DEV), torch.zeros(K.height, K.width, 4, device=DEV)
    T_ref = frames[5].pose @ scenes.perturbation(np.random.default_rng(8), 2.0, 0.02)
    gm.render(K, T_ref, rd, rn)
    ic.set_frame(cu(frames[5].depth), None, K, ZMIN, ZMAX, DSUP)
    T = torch.eye(4, dtype=torch.float64, device=DEV)
    ic.solve(rd, rn, K, T, dt.icp_opts(levels=3, eps=(0.02, 0.05, 0.1), lam=0.0))
    true = np.linalg.inv(T_ref) @ frames[5].pose
    E = np.linalg.inv(true) @ T.cpu().numpy()
    assert np.linalg.norm(E[:3, 3]) < 3e-3


def test_depth_mae_matches_oracle():
    rng = np.random.default_rng(5)
    for n in (0, 1, 1000, 307200, 1 << 21):
        a = (1.0 + rng.random(n)).astype(np.float32)
        b = (a + rng.normal(0, 0.01, n)).astype(np.float32)
        a[rng.random(n) < 0.1] = 0
        b[rng.random(n) < 0.1] = 0
        out = dt.depth_mae(cu(a), cu(b))
        torch.cuda.synchronize()
        s, c = out.cpu().numpy()
        so, co = OF.depth_mae(a, b)
        assert int(c) == co
        assert s == pytest.approx(so, rel=1e-12, abs=0.0)
