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
            # rows whose pixel and association are the same at both perturbed poses
            key = lambda R: {(a, b, c, d): i for i, (a, b, c, d) in enumerate(np.hstack([R.pix, R.ref]))}
            kp, km = key(rp), key(rm)
            both = [(i, kp[k], km[k]) for k, i in key(rows).items() if k in kp and k in km]
            assert len(both) >= 0.99 * rows.r.shape[0]
            i0, ip, im = (np.array(x) for x in zip(*both))
            fd = (rp.r[ip] - rm.r[im]) / (2 * h)
            assert np.allclose(fd, rows.J[i0, j], rtol=1e-6, atol=1e-7)


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


def test_pyramid_is_the_mean_of_valid_children():
    rng = np.random.default_rng(2)
    d = rng.uniform(0.5, 3.0, size=(48, 64)).astype(np.float32)
    d[rng.random(d.shape) < 0.3] = 0
    d64 = icp.downsample_depth(d.astype(np.float64))
    # brute force mean of valid children
    for v in range(24):
        for u in range(32):
            c = d[2 * v:2 * v + 2, 2 * u:2 * u + 2].astype(np.float64)
            c = c[c > 0]
            exp = c.mean() if c.size else 0.0
            assert d64[v, u] == pytest.approx(exp, rel=1e-15)


# ------------------------------------------- Levenberg-Marquardt (Sec. 7) ----

def _lm_problem(deg, m, seed):
    s, K, T_ref, T_cur, rd, rn, cur = _ref_and_current(deg, m, seed=seed)
    return icp.pyramid(cur.depth, K, 3), rd, rn, K, np.linalg.inv(T_ref) @ T_cur


@pytest.mark.parametrize("deg,m", [(2, 0.02), (5, 0.10)])
def test_lm_exact_recovery(deg, m):
    """LM reaches the true motion of noiseless planes (as Gauss-Newton does)."""
    levels, rd, rn, K, true = _lm_problem(deg, m, deg)
    st = icp.Settings(eps=(0.02, 0.2, 0.3), iters=(30, 15, 15), lm=True)
    dT, log = icp.track(levels, rd, rn, K, np.eye(4), st)
    E = np.linalg.inv(true) @ dT
    ang = np.arccos(np.clip((np.trace(E[:3, :3]) - 1) / 2, -1, 1))
    assert ang < 1e-6 and np.linalg.norm(E[:3, 3]) < 1e-6
    # a rejected evaluation never becomes the accepted one: accepted errors strictly decrease
    for lvl in range(3):
        acc = [e["E"] for e in log if e["level"] == lvl and e.get("accepted")]
        assert all(b < a for a, b in zip(acc, acc[1:]))


def test_lm_without_damping_is_gauss_newton():
    """mu = 0 (tau = 0) turns the damped system into the Gauss-Newton one: while every step is
    accepted the two schedules take identical steps."""
    levels, rd, rn, K, true = _lm_problem(2, 0.02, 3)
    gn = icp.Settings(eps=(0.02, 0.2, 0.3), iters=(3, 3, 3), stop=0.0)
    lm = icp.Settings(eps=(0.02, 0.2, 0.3), iters=(3, 3, 3), stop=0.0, lm=True, lm_tau=0.0)
    Tg, lg = icp.track(levels, rd, rn, K, np.eye(4), gn)
    Tl, ll = icp.track(levels, rd, rn, K, np.eye(4), lm)
    assert all(e["accepted"] for e in ll)
    assert np.array_equal(Tg, Tl)
    assert [e["E"] for e in lg] == [e["E"] for e in ll]


@pytest.mark.parametrize("tau", [1e-3, 1.0])
def test_lm_predicted_decrease_matches_near_linear_error(tau):
    """For a small motion the residuals are nearly linear in xi, so the quadratic model is
    nearly exact and the gain ratio of the first step is ~1. The predicted decrease must carry
    both xi^T H xi and the damping term 2 mu xi^T xi: with tau = 1 the damping term is a large
    part of it, and dropping it (or the factor 2 of g in E(xi)) moves rho far from 1."""
    levels, rd, rn, K, true = _lm_problem(0.2, 0.002, 5)
    # the full-resolution level alone: its points lie on the planes (no 2x2 means across creases)
    st = icp.Settings(eps=(0.02,), iters=(2,), stop=0.0, lm=True, lm_tau=tau)
    dT, log = icp.track(levels[:1], rd, rn, K, np.eye(4), st)
    first, second = log[0], log[1]
    assert abs(second["rho"] - 1.0) < 1e-3, second
    # Madsen's update for rho ~ 1: mu shrinks by the floor factor 1/3
    assert second["mu"] == pytest.approx(first["mu"] / 3.0, rel=1e-12)


def test_lm_rejections_grow_the_damping():
    """An evaluation with a larger error than the accepted one is rejected and mu grows by nu,
    which doubles on each further rejection (x2, x4, x8 ...) and returns to 2 on acceptance.
    Sensor noise makes the error stall near the optimum, where rejections occur."""
    import oracle
    s = scenes.planes_scene()
    rng = np.random.default_rng(2)
    T_ref = s.poses[0]
    cur = s.render(T_ref @ scenes.perturbation(rng, 2, 0.02), noise=True)
    ref = s.render(T_ref, noise=False, exact=True)
    rn = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    rn[..., :3] = ref.normals
    lv = icp.pyramid(oracle.preprocess(cur.depth, s.K, 0.1, 6.0, 0.02)["z"], s.K, 3)
    st = icp.Settings(eps=(0.02, 0.2, 0.3), iters=(10, 5, 4), lm=True)
    dT, log = icp.track(lv, ref.depth, rn, s.K, np.eye(4), st)
    log = [e for e in log if "mu" in e]
    assert sum(not e["accepted"] for e in log) >= 2
    nu = 2.0
    for a, b in zip(log, log[1:]):
        if b["level"] != a["level"]:
            nu = 2.0
            continue
        if b["accepted"]:
            r = b["rho"]
            assert r > 0 and b["mu"] == pytest.approx(a["mu"] * max(1 / 3, 1 - (2 * r - 1) ** 3), rel=1e-12)
            nu = 2.0
        else:
            assert b["rho"] <= 0 and b["mu"] == pytest.approx(a["mu"] * nu, rel=1e-12)
            nu *= 2.0
    for lvl in range(3):
        acc = [e["E"] for e in log if e["level"] == lvl and e["accepted"]]
        assert all(y < x for x, y in zip(acc, acc[1:]))


# ------------------------------------------ multi-sensor scale anchoring ----

CYCLE = (1.0, 1.05, 0.975, 1.025, 0.95)  # Sec. 6: five sensors, five consecutive frames each


def _cycle(n_cycles):
    sensor = np.repeat(np.tile(np.arange(5), n_cycles), 5)
    return sensor, np.log(np.array(CYCLE))[sensor]


def test_scale_anchor_is_the_papers_difference():
    """With a constant anchor estimate s^_0 and anchor value 0 the result is s^_i - s^_0 for every
    other sensor (Eq. scale_anchor in the log domain)."""
    sensor, true = _cycle(3)
    s0 = 0.0123
    est = np.where(sensor == 0, s0, true + 0.5)
    out = icp.scale_anchor(est, sensor, 0, 0.0)
    assert np.array_equal(out[sensor == 0], np.zeros(15))
    np.testing.assert_allclose(out[sensor != 0], (true + 0.5 - s0)[sensor != 0], rtol=0, atol=1e-15)


def test_scale_anchor_removes_common_drift():
    """Estimates = true log scale + a drift common to all sensors. Drift constant over each
    cycle cancels exactly; a linear drift leaves at most its change since the anchor's last frame
    (20 frames for the last sensor of a cycle)."""
    sensor, true = _cycle(4)
    cyc = np.arange(sensor.shape[0]) // 25
    est = true + 0.01 * cyc
    out = icp.scale_anchor(est, sensor, 0, np.log(CYCLE[0]))
    np.testing.assert_allclose(out, true, rtol=0, atol=1e-15)
    rate = 1e-4
    t = np.arange(sensor.shape[0])
    out = icp.scale_anchor(true + rate * t, sensor, 0, 0.0)
    last_anchor = np.array([max(j for j in range(k + 1) if sensor[j] == 0) for k in t])
    np.testing.assert_allclose(out - true, rate * (t - last_anchor), rtol=0, atol=1e-14)
    assert np.max(np.abs(out - true)) <= rate * 20 + 1e-14  # unanchored: rate * 99


def test_scale_anchor_before_the_first_anchor_frame():
    sensor = np.array([2, 3, 0, 2, 1])
    est = np.array([0.1, 0.2, 0.05, 0.13, -0.04])
    out = icp.scale_anchor(est, sensor, 0, 0.0)
    assert out[0] == 0.1 and out[1] == 0.2 and out[2] == 0.0
    assert out[3] == 0.13 - 0.05 and out[4] == -0.04 - 0.05


def test_library_scale_anchor_matches_oracle():
    """dtsdf_scale_anchor (host arithmetic in the library) equals the oracle bit for bit."""
    from paper_2301_12796_gb300 import build as B
    import paper_2301_12796_gb300 as dt
    B.build()
    rng = np.random.default_rng(4)
    sensor = rng.integers(0, 5, size=400).astype(np.int32)
    est = rng.normal(0, 0.05, size=400)
    for anchor, val in ((0, 0.0), (3, 0.02)):
        assert np.array_equal(dt.scale_anchor(est, sensor, anchor, val), icp.scale_anchor(est, sensor, anchor, val))
    assert dt.scale_anchor(np.zeros(0), np.zeros(0, np.int32)).shape == (0,)


def test_lm_recovers_depth_scale_in_sim3():
    """Levenberg-Marquardt in Sim(3) reaches the same exact optimum as Gauss-Newton: the inverse
    of a 1.0625 depth scale and the true motion."""
    scale = 1.0625
    s, K, T_ref, T_cur, rd, rn, cur = _ref_and_current(2, 0.02, seed=11, depth_scale=scale)
    levels = icp.pyramid(cur.depth, K, 3)
    st = icp.Settings(sim3=True, eps=(0.02, 0.2, 0.3), iters=(40, 20, 20), lm=True)
    dT, log = icp.track(levels, rd, rn, K, np.eye(4), st)
    true = np.linalg.inv(T_ref) @ T_cur
    s_est = np.cbrt(np.linalg.det(dT[:3, :3]))
    assert abs(s_est * scale - 1.0) < 1e-6
    R = dT[:3, :3] / s_est
    E = true[:3, :3].T @ R
    assert np.arccos(np.clip((np.trace(E) - 1) / 2, -1, 1)) < 1e-6
    assert np.linalg.norm(dT[:3, 3] - true[:3, 3]) < 1e-6


def _photometric_only(cl, kl, K, T_rs, thr=0.1, iters=15):
    dT = np.eye(4)
    for l in (2, 1, 0):
        for _ in range(iters):
            rows = icp.photometric_rows(cl[l], kl[l].I, K.scaled(l), T_rs, dT, thr, 1.0, 0.1, False)
            H, g, E, n = icp.normal_equations([rows])
            xi, ok = icp.solve(H, g)
            if not ok:
                return dT
            dT = icp.exp(xi) @ dT
    return dT


def test_photometric_only_schedule_recovers_known_motion():
    """Eq. keyframe_icp alone (no geometric rows) on a textured plane seen by a keyframe camera
    3 deg / 4 cm away from the render camera: Gauss-Newton from the identity recovers the
    current frame's 1 deg / 1 cm motion to the texture's interpolation limit. This fixes the
    direction of T_RS (render -> keyframe frame) and the sign of the residual and of its
    Jacobian: with T_RS inverted the schedule ends centimetres away."""
    s = scenes.plane_scene()
    K = scenes.Intrinsics(160, 120, 120.0, 120.0, 79.5, 59.5)
    T_ref = s.poses[0]
    rng = np.random.default_rng(11)
    T_kf = T_ref @ scenes.perturbation(rng, 3.0, 0.04)
    T_cur = T_ref @ scenes.perturbation(rng, 1.0, 0.01)
    cur = s.render(T_cur, K=K, noise=False)
    kf = s.render(T_kf, K=K, noise=False)
    T_rs = np.linalg.inv(T_kf) @ T_ref
    true = np.linalg.inv(T_ref) @ T_cur
    z = oracle.preprocess(cur.depth, K, 0.1, 6.0, 0.02)["z"]
    cl = icp.pyramid(z, K, 3, cur.rgb)
    kl = icp.pyramid(z, K, 3, kf.rgb)
    dT = _photometric_only(cl, kl, K, T_rs)
    ang = np.arccos(np.clip((np.trace(dT[:3, :3].T @ true[:3, :3]) - 1) / 2, -1, 1))
    assert np.linalg.norm(dT[:3, 3] - true[:3, 3]) < 2e-4 and ang < np.deg2rad(0.02)
    wrong = _photometric_only(cl, kl, K, np.linalg.inv(T_rs))
    assert np.linalg.norm(wrong[:3, 3] - true[:3, 3]) > 5e-3
