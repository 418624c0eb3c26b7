"""Pins of the oracle's ICP (Sec. 5, 5.2, 5.3, 6): exponential maps against closed
forms, Jacobians against finite differences, exact recovery of known motions."""
import numpy as np
import pytest

import oracle
from oracle import icp
import scenes


def rodrigues(w):
    th = np.linalg.norm(w)
    if th == 0:
        return np.eye(3)
    k = w / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx


def se3_V(w):
    th = np.linalg.norm(w)
    W = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    if th < 1e-8:
        return np.eye(3) + 0.5 * W
    return np.eye(3) + (1 - np.cos(th)) / th ** 2 * W + (th - np.sin(th)) / th ** 3 * W @ W


@pytest.mark.parametrize("scale", [1e-9, 1e-4, 0.3, 2.5])
def test_se3_exp_closed_form(scale):
    rng = np.random.default_rng(4)
    xi = rng.normal(size=6) * scale
    T = icp.exp(xi)
    assert np.allclose(T[:3, :3], rodrigues(xi[3:]), atol=1e-13)
    assert np.allclose(T[:3, 3], se3_V(xi[3:]) @ xi[:3], atol=1e-13)
    assert np.allclose(T[3], [0, 0, 0, 1])


@pytest.mark.parametrize("scale", [1e-9, 1e-3, 0.4])
def test_sim3_exp_structure(scale):
    rng = np.random.default_rng(5)
    xi = rng.normal(size=7) * scale
    S = icp.exp(xi)
    s = np.exp(xi[6])
    # upper block is e^sigma times the rotation exp(omega)
    assert np.allclose(S[:3, :3], s * rodrigues(xi[3:6]), atol=1e-13)
    # pure translation/scale: t = (e^sigma - 1)/sigma nu
    xt = np.zeros(7)
    xt[:3], xt[6] = xi[:3], xi[6]
    St = icp.exp(xt)
    fac = (np.exp(xi[6]) - 1) / xi[6]
    assert np.allclose(St[:3, 3], fac * xi[:3], rtol=1e-9)
    # group inverse
    assert np.allclose(icp.exp(xi) @ icp.exp(-xi), np.eye(4), atol=1e-12)
    assert np.allclose(icp.exp(0.3 * xi) @ icp.exp(0.7 * xi), S, atol=1e-12)


def _mask_edges(frame, r=2):
    """Zero the depth within r pixels of a crease or an occlusion edge, so that every
    association at the true pose pairs points of the same plane (zero residual)."""
    n, ids = frame.normals, frame.ids
    H, W = ids.shape
    bad = np.zeros((H, W), bool)
    for dv in range(-r, r + 1):
        for du in range(-r, r + 1):
            sv = slice(max(dv, 0), H + min(dv, 0))
            tv = slice(max(-dv, 0), H + min(-dv, 0))
            su = slice(max(du, 0), W + min(du, 0))
            tu = slice(max(-du, 0), W + min(-du, 0))
            diff = (ids[sv, su] != ids[tv, tu]) | (np.sum(n[sv, su] * n[tv, tu], -1) < 1 - 1e-9)
            bad[tv, tu] |= diff
    d = frame.depth.copy()
    d[bad] = 0
    return d


def _ref_and_current(perturb_deg, perturb_m, seed=0, depth_scale=1.0, K=None):
    s = scenes.planes_scene()
    K = K or s.K
    T_ref = s.poses[0]
    rng = np.random.default_rng(seed)
    P = scenes.perturbation(rng, perturb_deg, perturb_m)
    T_cur = T_ref @ P
    ref = s.render(T_ref, K=K, noise=False, exact=True)
    cur = s.render(T_cur, K=K, noise=False, depth_scale=depth_scale, exact=True)
    cur.depth = _mask_edges(cur)
    ref_depth = _mask_edges(ref)
    ref_normals = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    ref_normals[..., :3] = ref.normals
    return s, K, T_ref, T_cur, ref_depth, ref_normals, cur


def test_geometric_jacobian_matches_finite_differences():
    s, K, T_ref, T_cur, rd, rn, cur = _ref_and_current(2, 0.02)
    lv = icp.pyramid(cur.depth, K, 1)[0]
    dT = np.linalg.inv(T_ref) @ T_cur @ icp.exp(np.array([0.003, -0.002, 0.001, 0.002, 0.001, -0.003]))
    for sim3 in (False, True):
        rows = icp.geometric_rows(lv, rd, rn, K, dT, 0.05, 0.1, sim3)
        k = 7 if sim3 else 6
        h = 1e-7
        for j in range(k):
            e = np.zeros(k)
            e[j] = h
            # fixed association: recompute x with the perturbed pose at the same pixels
            rp = icp.geometric_rows(lv, rd, rn, K, icp.exp(e) @ dT, 0.05, 0.1, sim3)
            rm = icp.geometric_rows(lv, rd, rn, K, icp.exp(-e) @ dT, 0.05, 0.1, sim3)
            if rp.r.shape != rows.r.shape or rm.r.shape != rows.r.shape:
                continue
            fd = (rp.r - rm.r) / (2 * h)
            assert np.allclose(fd, rows.J[:, j], rtol=1e-6, atol=1e-7)


def test_photometric_jacobian_matches_finite_differences():
    s = scenes.planes_scene()
    K = s.K
    T_ref = s.poses[0]
    rng = np.random.default_rng(9)
    T_kf = T_ref @ scenes.perturbation(rng, 3, 0.03)
    T_cur = T_ref @ scenes.perturbation(rng, 1, 0.01)
    cur = s.render(T_cur, noise=False)
    lv = icp.pyramid(cur.depth, K, 1, cur.rgb)[0]
    # an affine keyframe image: central differences and bilinear interpolation are then exact,
    # so the analytic Jacobian must equal the finite-difference derivative of the residual
    vv, uu = np.mgrid[0:K.height, 0:K.width]
    kf_I = 0.3 + 0.002 * uu + 0.0013 * vv
    T_rs = np.linalg.inv(T_kf) @ T_ref
    dT = np.linalg.inv(T_ref) @ T_cur
    for sim3 in (False, True):
        rows = icp.photometric_rows(lv, kf_I, K, T_rs, dT, 10.0, 0.1, 0.1, sim3)
        k = 7 if sim3 else 6
        h = 1e-7
        agree = []
        for j in range(k):
            e = np.zeros(k)
            e[j] = h
            rp = icp.photometric_rows(lv, kf_I, K, T_rs, icp.exp(e) @ dT, 10.0, 0.1, 0.1, sim3)
            rm = icp.photometric_rows(lv, kf_I, K, T_rs, icp.exp(-e) @ dT, 10.0, 0.1, 0.1, sim3)
            assert rp.r.shape == rows.r.shape == rm.r.shape
            fd = (rp.r - rm.r) / (2 * h)
            agree.append(np.isclose(fd, rows.J[:, j], rtol=1e-6, atol=1e-8))
        assert np.all(np.stack(agree)), np.mean(np.stack(agree))


@pytest.mark.parametrize("deg,m", [(2, 0.02), (5, 0.10)])
def test_se3_exact_recovery(deg, m):
    s, K, T_ref, T_cur, rd, rn, cur = _ref_and_current(deg, m, seed=deg)
    levels = icp.pyramid(cur.depth, K, 3)
    st = icp.Settings(eps=(0.02, 0.2, 0.3), iters=(30, 15, 15))
    dT, log = icp.track(levels, rd, rn, K, np.eye(4), st)
    true = np.linalg.inv(T_ref) @ T_cur
    E = np.linalg.inv(true) @ dT
    ang = np.arccos(np.clip((np.trace(E[:3, :3]) - 1) / 2, -1, 1))
    assert ang < 1e-6 and np.linalg.norm(E[:3, 3]) < 1e-6


def test_sim3_recovers_depth_scale():
    scale = 1.0625
    s, K, T_ref, T_cur, rd, rn, cur = _ref_and_current(2, 0.02, seed=11, depth_scale=scale)
    levels = icp.pyramid(cur.depth, K, 3)
    st = icp.Settings(sim3=True, eps=(0.02, 0.2, 0.3), iters=(40, 20, 20))
    dT, log = icp.track(levels, rd, rn, K, np.eye(4), st)
    true = np.linalg.inv(T_ref) @ T_cur
    s_est = np.cbrt(np.linalg.det(dT[:3, :3]))
    assert abs(s_est * scale - 1.0) < 1e-6
    R = dT[:3, :3] / s_est
    E = true[:3, :3].T @ R
    assert np.arccos(np.clip((np.trace(E) - 1) / 2, -1, 1)) < 1e-6
    assert np.linalg.norm(dT[:3, 3] - true[:3, 3]) < 1e-6


def test_sim3_single_plane_is_degenerate():
    s = scenes.plane_scene()
    T = s.poses[0]
    ref = s.render(T, noise=False, exact=True)
    rn = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    rn[..., :3] = ref.normals
    lv = icp.pyramid(ref.depth, s.K, 1)[0]
    st = icp.Settings(sim3=True)
    out = icp.step(lv, ref.depth, rn, s.K, np.eye(4), 0.05, st)
    assert out[-1] is False


def test_pyramid_single_and_double_precision_agree():
    rng = np.random.default_rng(2)
    d = rng.uniform(0.5, 3.0, size=(48, 64)).astype(np.float32)
    d[rng.random(d.shape) < 0.3] = 0
    d32, d64 = icp.downsample_depth(d, d.astype(np.float64))
    # brute force mean of valid children
    for v in range(24):
        for u in range(32):
            c = d[2 * v:2 * v + 2, 2 * u:2 * u + 2].astype(np.float64)
            c = c[c > 0]
            exp = c.mean() if c.size else 0.0
            assert d64[v, u] == pytest.approx(exp, rel=1e-15)
            assert d32[v, u] == pytest.approx(exp, rel=1e-6)
