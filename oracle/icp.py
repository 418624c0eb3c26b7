"""FP64 oracle of the point-to-plane ICP in SE(3) and Sim(3), with the
frame-to-keyframe photometric rows (test infrastructure only; see package doc).

Paper passages followed (Splietker & Behnke):
  * Eq. geometric_ICP / Eq. ICP_geometric_dx: r_i = <q_i - exp(xi) dT p_i, n_i>,
    J_i = (-n_i, -(dT p_i) x n_i) with xi = (nu, omega).
  * Eq. sim3_derivative: the Sim(3) point derivative [I, -(x)^, x] adds the 7th
    column -<n_i, x_i>.
  * Eq. ICP_Hessian / Eq. ICP_solution / Eq. deltaT_update: H = sum w J J^T,
    g = sum w J r (the common factor 2 cancels in H xi = -g), Cholesky solve,
    dT <- exp(xi) dT; stop when ||xi|| < 1e-6 (Sec. 8 ICP settings).
  * Eq. ICP_weight: w = 1 / (z + (1 - z_min))^2.
  * Eq. combined_icp with lambda = 0.1 (not squared) and the depth weight on the
    photometric rows; Eq. keyframe_icp: r = I_cur(u) - I_kf(pi(K T_RS exp(xi) dT p)).
    Its printed derivative drops the minus sign of r and has the sign of x/z^2
    flipped; this oracle uses the exact derivative of the defined residual,
    J = -grad I_kf^T d(pi)/dy R_RS [I | -x^ (| x)], checked by finite differences.
  * Sim(3) exponential: the matrix exponential of the 4x4 generator
    [[omega^ + sigma I, nu], [0, 0]] (the paper prints the block form with an
    undefined V; the matrix exponential fixes V).
  * Sec. 7 / Sec. 8: 3-level pyramid (2x2 mean of valid depths, intrinsics
    f/2, (c - 0.5)/2), association by projecting the current point into the
    full-resolution render and rounding to the nearest pixel, distance outlier
    threshold 0.05 m coarse / 0.005 m finest, intensity threshold 0.175 / 0.05.

Decisions (pixel association, inlier distance, image bounds) are taken in
single precision with the kernel's operation order: x = p + ((A p) + t) with
A = sR - I. Values are computed in double.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg

F32 = np.float32


# ----------------------------------------------------------------- Lie ----

def hat(w) -> np.ndarray:
    """Eq. wedge_operator."""
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def generator(xi) -> np.ndarray:
    """4x4 generator of xi = (nu, omega[, sigma])."""
    xi = np.asarray(xi, np.float64)
    G = np.zeros((4, 4))
    sigma = xi[6] if xi.shape[0] == 7 else 0.0
    G[:3, :3] = hat(xi[3:6]) + sigma * np.eye(3)
    G[:3, 3] = xi[0:3]
    return G


def exp(xi) -> np.ndarray:
    """Exponential map se(3)/sim(3) -> SE(3)/Sim(3): matrix exponential of the generator."""
    return scipy.linalg.expm(generator(xi))


# ------------------------------------------------------------- images -----

def intensity(rgb: np.ndarray) -> np.ndarray:
    """I = (0.299 R + 0.587 G + 0.114 B) / 255 in double."""
    c = rgb.astype(np.float64)
    return (0.299 * c[..., 0] + 0.587 * c[..., 1] + 0.114 * c[..., 2]) / 255.0


def intensity_f32(rgb: np.ndarray) -> np.ndarray:
    c = rgb.astype(F32)
    return ((F32(0.299) * c[..., 0] + F32(0.587) * c[..., 1]) + F32(0.114) * c[..., 2]) / F32(255.0)


def downsample_depth(d32: np.ndarray, d64: np.ndarray):
    """2x2 mean of the valid (> 0) children, in the child order (0,0),(1,0),(0,1),(1,1).
    Single precision (sum in that order, then divide by the count) and double."""
    H, W = d32.shape[0] // 2, d32.shape[1] // 2
    s32 = np.zeros((H, W), F32)
    s64 = np.zeros((H, W))
    n = np.zeros((H, W), np.int32)
    for dy, dx in ((0, 0), (0, 1), (1, 0), (1, 1)):
        c32 = d32[dy:2 * H:2, dx:2 * W:2]
        c64 = d64[dy:2 * H:2, dx:2 * W:2]
        v = c32 > 0
        s32 = np.where(v, (s32 + c32).astype(F32), s32)
        s64 = np.where(v, s64 + c64, s64)
        n += v
    out32 = np.where(n > 0, s32 / np.maximum(n, 1).astype(F32), F32(0)).astype(F32)
    out64 = np.where(n > 0, s64 / np.maximum(n, 1), 0.0)
    return out32, out64


def downsample_mean(img: np.ndarray) -> np.ndarray:
    H, W = img.shape[0] // 2, img.shape[1] // 2
    return 0.25 * (img[0:2 * H:2, 0:2 * W:2] + img[0:2 * H:2, 1:2 * W:2] + img[1:2 * H:2, 0:2 * W:2]
                   + img[1:2 * H:2, 1:2 * W:2])


def grad_image(I: np.ndarray):
    """Central differences / 2; zero on the one-pixel border."""
    gx = np.zeros_like(I)
    gy = np.zeros_like(I)
    gx[:, 1:-1] = 0.5 * (I[:, 2:] - I[:, :-2])
    gy[1:-1, :] = 0.5 * (I[2:, :] - I[:-2, :])
    return gx, gy


@dataclass
class Level:
    d32: np.ndarray
    d64: np.ndarray
    K: object
    I: np.ndarray | None = None


def pyramid(depth_filtered: np.ndarray, K, levels: int, rgb: np.ndarray | None = None) -> list[Level]:
    """Levels 0..levels-1 of the current frame. ``depth_filtered`` is the
    outlier-filtered depth (Sec. 7)."""
    d32 = np.ascontiguousarray(depth_filtered, F32)
    d64 = d32.astype(np.float64)
    I = None if rgb is None else intensity(rgb)
    out = [Level(d32, d64, K, I)]
    for _ in range(1, levels):
        d32, d64 = downsample_depth(d32, d64)
        I = None if I is None else downsample_mean(I)
        out.append(Level(d32, d64, out[-1].K.scaled(1), I))
    return out


# -------------------------------------------------------- association -----

def _backproject32(z32, K):
    H, W = z32.shape
    u = np.arange(W, dtype=F32)[None, :]
    v = np.arange(H, dtype=F32)[:, None]
    a = (u - F32(K.cx)) / F32(K.fx)
    b = (v - F32(K.cy)) / F32(K.fy)
    return np.stack([(z32 * a).astype(F32), (z32 * b).astype(F32), z32], axis=-1)


def _backproject64(z64, K):
    H, W = z64.shape
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    return np.stack([z64 * ((u - K.cx) / K.fx), z64 * ((v - K.cy) / K.fy), z64], axis=-1)


def _transform32(dT: np.ndarray, p32: np.ndarray):
    """delta = (A p) + t with A = (sR - I) in single precision, x = p + delta."""
    A = (dT[:3, :3] - np.eye(3)).astype(F32)
    t = dT[:3, 3].astype(F32)
    d = [(((A[a, 0] * p32[..., 0]).astype(F32) + (A[a, 1] * p32[..., 1]).astype(F32)).astype(F32)
          + (A[a, 2] * p32[..., 2]).astype(F32)).astype(F32) for a in range(3)]
    delta = np.stack([(d[a] + t[a]).astype(F32) for a in range(3)], axis=-1)
    return (p32 + delta).astype(F32)


@dataclass
class Rows:
    J: np.ndarray    # N x 6|7
    r: np.ndarray    # N
    w: np.ndarray    # N
    n_geo: int
    n_photo: int


def geometric_rows(level: Level, ref_depth32: np.ndarray, ref_normals32: np.ndarray, K_ref, dT: np.ndarray,
                   eps: float, z_min: float, sim3: bool) -> Rows:
    """Point-to-plane rows (Eq. geometric_ICP, Eq. ICP_geometric_dx, Eq. sim3_derivative,
    Eq. ICP_weight) for the pixels of one pyramid level."""
    z32 = level.d32
    p32 = _backproject32(z32, level.K)
    x32 = _transform32(dT, p32)
    Hr, Wr = ref_depth32.shape
    valid = z32 > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        zpos = x32[..., 2] > 0
        uf = ((x32[..., 0] / x32[..., 2]).astype(F32) * F32(K_ref.fx)).astype(F32) + F32(K_ref.cx)
        vf = ((x32[..., 1] / x32[..., 2]).astype(F32) * F32(K_ref.fy)).astype(F32) + F32(K_ref.cy)
        ur = np.floor((uf + F32(0.5)).astype(F32))
        vr = np.floor((vf + F32(0.5)).astype(F32))
    inb = valid & zpos & (ur >= 0) & (vr >= 0) & (ur < Wr) & (vr < Hr)
    ui = np.where(inb, ur, 0).astype(np.int64)
    vi = np.where(inb, vr, 0).astype(np.int64)
    dr32 = np.where(inb, ref_depth32[vi, ui], F32(0))
    ok = inb & (dr32 > 0)
    ar = ((ui.astype(F32) - F32(K_ref.cx)) / F32(K_ref.fx)).astype(F32)
    br = ((vi.astype(F32) - F32(K_ref.cy)) / F32(K_ref.fy)).astype(F32)
    q32 = np.stack([(dr32 * ar).astype(F32), (dr32 * br).astype(F32), dr32], axis=-1)
    e = (q32 - x32).astype(F32)
    d2 = (((e[..., 0] * e[..., 0]).astype(F32) + (e[..., 1] * e[..., 1]).astype(F32)).astype(F32)
          + (e[..., 2] * e[..., 2]).astype(F32)).astype(F32)
    ok &= d2 <= F32(eps) * F32(eps)
    # values in double
    idx = np.nonzero(ok)
    p = _backproject64(level.d64, level.K)[idx]
    x = p @ dT[:3, :3].T + dT[:3, 3]
    dr = dr32[idx].astype(np.float64)
    uu, vv = ui[idx].astype(np.float64), vi[idx].astype(np.float64)
    q = np.stack([dr * ((uu - K_ref.cx) / K_ref.fx), dr * ((vv - K_ref.cy) / K_ref.fy), dr], axis=-1)
    n = ref_normals32[vi[idx], ui[idx], :3].astype(np.float64)
    r = np.einsum("ij,ij->i", q - x, n)
    cols = [-n, -np.cross(x, n)]
    if sim3:
        cols.append(-np.einsum("ij,ij->i", n, x)[:, None])
    J = np.concatenate(cols, axis=1)
    z = level.d64[idx]
    w = 1.0 / (z + (1.0 - z_min)) ** 2
    return Rows(J, r, w, J.shape[0], 0)


def bilinear(img: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    u0 = np.floor(u).astype(np.int64)
    v0 = np.floor(v).astype(np.int64)
    a = u - u0
    b = v - v0
    return ((1 - a) * (1 - b) * img[v0, u0] + a * (1 - b) * img[v0, u0 + 1] + (1 - a) * b * img[v0 + 1, u0]
            + a * b * img[v0 + 1, u0 + 1])


def photometric_rows(level: Level, kf_I: np.ndarray, K_kf, T_rs: np.ndarray, dT: np.ndarray, thr: float,
                     lam: float, z_min: float, sim3: bool) -> Rows:
    """Frame-to-keyframe photometric rows (Eq. keyframe_icp, Eq. combined_icp).

    kf_I: keyframe intensity at this level; K_kf: its intrinsics; T_rs: transform
    from the render camera frame to the keyframe camera frame."""
    z32 = level.d32
    p32 = _backproject32(z32, level.K)
    x32 = _transform32(dT, p32)
    Rf = T_rs[:3, :3].astype(F32)
    tf = T_rs[:3, 3].astype(F32)
    y32 = np.stack([(((Rf[a, 0] * x32[..., 0]).astype(F32) + (Rf[a, 1] * x32[..., 1]).astype(F32)).astype(F32)
                     + (Rf[a, 2] * x32[..., 2]).astype(F32) + tf[a]).astype(F32) for a in range(3)], axis=-1)
    Hk, Wk = kf_I.shape
    valid = z32 > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        zpos = y32[..., 2] > 0
        uk = ((y32[..., 0] / y32[..., 2]).astype(F32) * F32(K_kf.fx)).astype(F32) + F32(K_kf.cx)
        vk = ((y32[..., 1] / y32[..., 2]).astype(F32) * F32(K_kf.fy)).astype(F32) + F32(K_kf.cy)
    ok = valid & zpos & (uk >= 1) & (vk >= 1) & (uk < Wk - 2) & (vk < Hk - 2)
    idx = np.nonzero(ok)
    p = _backproject64(level.d64, level.K)[idx]
    x = p @ dT[:3, :3].T + dT[:3, 3]
    y = x @ T_rs[:3, :3].T + T_rs[:3, 3]
    # sampling position in double; the single-precision path only decided the bounds
    us = K_kf.fx * y[:, 0] / y[:, 2] + K_kf.cx
    vs = K_kf.fy * y[:, 1] / y[:, 2] + K_kf.cy
    us = np.clip(us, 1.0, Wk - 2 - 1e-9)
    vs = np.clip(vs, 1.0, Hk - 2 - 1e-9)
    gx, gy = grad_image(kf_I)
    Ik = bilinear(kf_I, us, vs)
    gxs = bilinear(gx, us, vs)
    gys = bilinear(gy, us, vs)
    r = level.I[idx] - Ik
    keep = np.abs(r) <= thr
    y, x, r, gxs, gys = y[keep], x[keep], r[keep], gxs[keep], gys[keep]
    z = level.d64[idx][keep]
    X, Y, Z = y[:, 0], y[:, 1], y[:, 2]
    # d(pi)/dy in pixels, rows (u, v)
    dpi = np.zeros((y.shape[0], 2, 3))
    dpi[:, 0, 0] = K_kf.fx / Z
    dpi[:, 0, 2] = -K_kf.fx * X / Z ** 2
    dpi[:, 1, 1] = K_kf.fy / Z
    dpi[:, 1, 2] = -K_kf.fy * Y / Z ** 2
    gI = np.stack([gxs, gys], axis=-1)                      # N x 2
    a = -np.einsum("ni,nij->nj", gI, dpi) @ T_rs[:3, :3]    # N x 3  (d r / d x in render frame)
    cols = [a, np.cross(x, a)]                               # a . (-x^ e_k) = (x x a)_k
    if sim3:
        cols.append(np.einsum("ij,ij->i", a, x)[:, None])
    J = np.concatenate(cols, axis=1)
    w = lam / (z + (1.0 - z_min)) ** 2
    return Rows(J, r, w, 0, J.shape[0])


def normal_equations(rows: list[Rows]):
    """Eq. ICP_Hessian without the common factor 2: H = J^T W J, g = J^T W r."""
    J = np.concatenate([x.J for x in rows])
    r = np.concatenate([x.r for x in rows])
    w = np.concatenate([x.w for x in rows])
    H = J.T @ (w[:, None] * J)
    g = J.T @ (w * r)
    E = float(np.sum(w * r * r))
    n = int(sum(x.n_geo + x.n_photo for x in rows))
    return H, g, E, n


DEGENERATE_PIVOT = 1e-10


def solve(H: np.ndarray, g: np.ndarray):
    """Eq. ICP_solution by Cholesky. Returns (xi, ok). A pivot below
    1e-10 * max diag(H) is a rank-deficient (degenerate) system."""
    k = H.shape[0]
    dmax = float(np.max(np.diag(H))) if k else 0.0
    if not dmax > 0:
        return np.zeros(k), False
    try:
        L = np.linalg.cholesky(H)
    except np.linalg.LinAlgError:
        return np.zeros(k), False
    if np.min(np.diag(L) ** 2) <= DEGENERATE_PIVOT * dmax:
        return np.zeros(k), False
    y = scipy.linalg.solve_triangular(L, -g, lower=True)
    xi = scipy.linalg.solve_triangular(L.T, y, lower=False)
    return xi, True


@dataclass
class Settings:
    sim3: bool = False
    eps: tuple = (0.005, 0.05, 0.05)          # per level, finest first
    iters: tuple = (10, 5, 4)                 # per level, finest first
    photo_thr: tuple = (0.05, 0.175, 0.175)
    lam: float = 0.1
    z_min: float = 0.1
    stop: float = 1e-6
    min_rows: int = 10
    lm: bool = False  # Levenberg-Marquardt with Madsen's damping update instead of Gauss-Newton
    lm_tau: float = 1e-3  # initial damping mu = lm_tau * max diag(H) of a level's first evaluation


def step(level: Level, ref_depth32, ref_normals32, K_ref, dT, eps, settings: Settings, photo=None,
         level_index: int = 0):
    """One Gauss-Newton iteration. photo = (kf_I, K_kf, T_rs) or None.
    Returns (new dT, H, g, E, N, xi, ok)."""
    rows = [geometric_rows(level, ref_depth32, ref_normals32, K_ref, dT, eps, settings.z_min, settings.sim3)]
    if photo is not None:
        kf_I, K_kf, T_rs = photo
        rows.append(photometric_rows(level, kf_I, K_kf, T_rs, dT, settings.photo_thr[level_index], settings.lam,
                                     settings.z_min, settings.sim3))
    H, g, E, n = normal_equations(rows)
    if n < settings.min_rows:
        return dT, H, g, E, n, np.zeros(H.shape[0]), False
    xi, ok = solve(H, g)
    if not ok:
        return dT, H, g, E, n, xi, False
    return exp(xi) @ dT, H, g, E, n, xi, True


def lm_level(level: Level, ref_depth32, ref_normals32, K_ref, dT, eps, settings: Settings, iters: int, photo,
             level_index: int, log: list):
    """One pyramid level of Levenberg-Marquardt (Sec. 7: the implementation solves with LM and
    Madsen's damping update). Each iteration evaluates the rows at the current pose; the first
    evaluation is accepted and sets mu = tau max diag(H) (tau = settings.lm_tau, 1e-3), nu = 2; later ones are accepted when
    the gain ratio rho = (E_acc - E) / (predicted decrease) is positive (mu <- mu max(1/3,
    1 - (2 rho - 1)^3), nu <- 2), otherwise the pose returns to the accepted one and mu <- mu nu,
    nu <- 2 nu. The step solves (H_acc + mu I) xi = -g_acc; its predicted decrease of E is
    xi^T H_acc xi + 2 mu xi^T xi (E(xi) ~ E + 2 g^T xi + xi^T H xi in the convention without the
    factor 2); the pose becomes exp(xi) dT_acc. The level stops at ||xi|| < stop."""
    acc = None
    mu = nu = pred = 0.0
    for it in range(iters):
        rows = [geometric_rows(level, ref_depth32, ref_normals32, K_ref, dT, eps, settings.z_min, settings.sim3)]
        if photo is not None:
            kf_I, K_kf, T_rs = photo
            rows.append(photometric_rows(level, kf_I, K_kf, T_rs, dT, settings.photo_thr[level_index], settings.lam,
                                         settings.z_min, settings.sim3))
        H, g, E, n = normal_equations(rows)
        if n < settings.min_rows:
            log.append(dict(level=level_index, it=it, E=E, n=n, step=0.0, ok=False))
            break
        if acc is None:
            mu, nu = settings.lm_tau * float(np.max(np.diag(H))), 2.0
            acc = (dT, H, g, E)
            accepted, rho = True, None
        else:
            rho = (acc[3] - E) / pred
            accepted = rho > 0
            if accepted:
                mu *= max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)
                nu = 2.0
                acc = (dT, H, g, E)
            else:
                mu *= nu
                nu *= 2.0
                dT = acc[0]
        Ha, ga = acc[1], acc[2]
        xi, ok = solve(Ha + mu * np.eye(Ha.shape[0]), ga)
        if not ok:
            log.append(dict(level=level_index, it=it, E=E, n=n, step=0.0, ok=False, accepted=accepted))
            break
        pred = float(xi @ Ha @ xi + 2.0 * mu * (xi @ xi))
        dT = exp(xi) @ acc[0]
        log.append(dict(level=level_index, it=it, E=E, n=n, step=float(np.linalg.norm(xi)), ok=True,
                        accepted=accepted, mu=mu, rho=rho, pred=pred))
        if np.linalg.norm(xi) < settings.stop:
            break
    return dT


def track(levels: list[Level], ref_depth32, ref_normals32, K_ref, dT0, settings: Settings, photo_levels=None):
    """Coarse-to-fine schedule: levels from coarsest to finest, iters[l] each,
    stopping a level when ||xi|| < settings.stop. photo_levels[l] = (kf_I, K_kf, T_rs).
    settings.lm selects Levenberg-Marquardt (lm_level) instead of Gauss-Newton."""
    dT = np.array(dT0, np.float64)
    log = []
    if settings.lm:
        for l in reversed(range(len(levels))):
            photo = None if photo_levels is None else photo_levels[l]
            dT = lm_level(levels[l], ref_depth32, ref_normals32, K_ref, dT, settings.eps[l], settings,
                          settings.iters[l], photo, l, log)
        return dT, log
    for l in reversed(range(len(levels))):
        for it in range(settings.iters[l]):
            photo = None if photo_levels is None else photo_levels[l]
            dT, H, g, E, n, xi, ok = step(levels[l], ref_depth32, ref_normals32, K_ref, dT, settings.eps[l],
                                           settings, photo, l)
            log.append(dict(level=l, it=it, E=E, n=n, step=float(np.linalg.norm(xi)), ok=ok))
            if not ok or np.linalg.norm(xi) < settings.stop:
                break
    return dT, log


# ------------------------------------------------- multi-sensor scale ----

def scale_anchor(log_scale_est, sensor, anchor: int = 0, anchor_value: float = 0.0) -> np.ndarray:
    """Sec. 6, Eq. scale_anchor, in the log domain (the printed equation equates a ratio of
    exponentials with a difference of logs; the difference of log scales is taken). Frames in
    time order; log_scale_est[k] is the log scale of frame k's Sim(3) estimate against the model.
    Scale drift of the model is common to all sensors, so the anchor sensor - whose scale is held
    at exp(anchor_value) - measures it: a frame of another sensor is compensated by the anchor's
    latest estimate, s_k = s^_k - (s^_anchor - anchor_value); the anchor's own frames get
    anchor_value; frames before the anchor's first estimate are left as estimated."""
    est = np.asarray(log_scale_est, np.float64)
    out = np.empty_like(est)
    latest = None
    for k in range(est.shape[0]):
        if int(sensor[k]) == anchor:
            latest = est[k]
            out[k] = anchor_value
        elif latest is None:
            out[k] = est[k]
        else:
            out[k] = est[k] - (latest - anchor_value)
    return out
