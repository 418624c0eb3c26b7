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

Every value and every decision (pixel association, inlier distance, image bounds,
intensity threshold) is computed in double precision. A decision within a stated
margin of its threshold is a tie: the rounding floor(x + 1/2) of a projected pixel
coordinate within TIE_PX = 2e-3 px of a half-integer (about 10x the single-precision
rounding of f x / z at f = 910), a camera depth within TIE_X = 1e-5 m of zero, the
inlier distance within TIE_X of eps, an image-bound test within TIE_PX, and an
intensity residual within 1e-6 + TIE_PX |grad I| of its threshold. ``Rows`` reports
the number of tie pixels and, for the normal equations, a bound on how much the
other outcomes of those decisions could change H and g (``tie_H``: Frobenius norm,
``tie_g``: per component), so that a comparison with an implementation that decides in
single precision can allow exactly that.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg

TIE_PX = 2e-3
TIE_X = 1e-5


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


def downsample_depth(d64: np.ndarray) -> np.ndarray:
    """2x2 mean of the valid (> 0) children (Sec. 7 pyramid)."""
    H, W = d64.shape[0] // 2, d64.shape[1] // 2
    s = np.zeros((H, W))
    n = np.zeros((H, W), np.int32)
    for dy, dx in ((0, 0), (0, 1), (1, 0), (1, 1)):
        c = d64[dy:2 * H:2, dx:2 * W:2]
        v = c > 0
        s = np.where(v, s + c, s)
        n += v
    return np.where(n > 0, s / np.maximum(n, 1), 0.0)


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
    d64: np.ndarray
    K: object
    I: np.ndarray | None = None


def pyramid(depth_filtered: np.ndarray, K, levels: int, rgb: np.ndarray | None = None) -> list[Level]:
    """Levels 0..levels-1 of the current frame. ``depth_filtered`` is the
    outlier-filtered depth (Sec. 7)."""
    d64 = np.asarray(depth_filtered, np.float64)
    I = None if rgb is None else intensity(rgb)
    out = [Level(d64, K, I)]
    for _ in range(1, levels):
        d64 = downsample_depth(d64)
        I = None if I is None else downsample_mean(I)
        out.append(Level(d64, out[-1].K.scaled(1), I))
    return out


# -------------------------------------------------------- association -----

def _backproject64(z64, K):
    H, W = z64.shape
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    return np.stack([z64 * ((u - K.cx) / K.fx), z64 * ((v - K.cy) / K.fy), z64], axis=-1)


def _round_alt(x):
    """floor(x + 1/2) and the other integer it could round to when x + 1/2 is within TIE_PX of
    an integer (else the same value)."""
    s = x + 0.5
    fl = np.floor(s)
    lo = (s - fl) < TIE_PX
    hi = (fl + 1.0 - s) < TIE_PX
    alt = np.where(lo, fl - 1.0, np.where(hi, fl + 1.0, fl))
    return fl, alt


@dataclass
class Rows:
    J: np.ndarray    # N x 6|7
    r: np.ndarray    # N
    w: np.ndarray    # N
    n_geo: int
    n_photo: int
    n_tie: int = 0                    # pixels with a tie decision
    tie_H: float = 0.0                # bound on |dH|_F from their other outcomes
    tie_g: np.ndarray | None = None   # bound on |dg| per component
    tie_E: float = 0.0                # bound on |dE|
    pix: np.ndarray | None = None     # N x 2 (v, u): the current-level pixel of each row
    ref: np.ndarray | None = None     # N x 2 (v, u): the associated render pixel (geometric rows)


def _contrib(J, r, w):
    """(w J J^T, w J r, w r^2) of single rows; J: k x d."""
    return w[:, None, None] * J[:, :, None] * J[:, None, :], (w * r)[:, None] * J, w * r * r


def _geo_row(x, q, n, z, z_min, sim3):
    r = np.einsum("ij,ij->i", q - x, n)
    cols = [-n, -np.cross(x, n)]
    if sim3:
        cols.append(-np.einsum("ij,ij->i", n, x)[:, None])
    J = np.concatenate(cols, axis=1)
    w = 1.0 / (z + (1.0 - z_min)) ** 2
    return J, r, w


def geometric_rows(level: Level, ref_depth32: np.ndarray, ref_normals32: np.ndarray, K_ref, dT: np.ndarray,
                   eps: float, z_min: float, sim3: bool) -> Rows:
    """Point-to-plane rows (Eq. geometric_ICP, Eq. ICP_geometric_dx, Eq. sim3_derivative,
    Eq. ICP_weight) for the pixels of one pyramid level: x = dT p is projected with the
    render intrinsics and rounded to the nearest pixel q (reading C11); the row exists when
    both depths are valid and |q - x| <= eps."""
    z = level.d64
    p = _backproject64(z, level.K)
    x = p @ dT[:3, :3].T + dT[:3, 3]
    Hr, Wr = ref_depth32.shape
    dref = ref_depth32.astype(np.float64)
    nref = ref_normals32[..., :3].astype(np.float64)
    valid = z > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        zpos = x[..., 2] > 0
        uf = (x[..., 0] / x[..., 2]) * K_ref.fx + K_ref.cx
        vf = (x[..., 1] / x[..., 2]) * K_ref.fy + K_ref.cy
        ur, ua = _round_alt(np.where(zpos, uf, -1e9))
        vr, va = _round_alt(np.where(zpos, vf, -1e9))

    def assoc(uu, vv):
        inb = valid & zpos & (uu >= 0) & (vv >= 0) & (uu < Wr) & (vv < Hr)
        ui = np.where(inb, uu, 0).astype(np.int64)
        vi = np.where(inb, vv, 0).astype(np.int64)
        dr = np.where(inb, dref[vi, ui], 0.0)
        q = np.stack([dr * ((ui - K_ref.cx) / K_ref.fx), dr * ((vi - K_ref.cy) / K_ref.fy), dr], axis=-1)
        dist = np.linalg.norm(q - x, axis=-1)
        ok = inb & (dr > 0)
        return ok & (dist <= eps), ok & (np.abs(dist - eps) < TIE_X), ui, vi, q

    ok, near, ui, vi, q = assoc(ur, vr)
    idx = np.nonzero(ok)
    J, r, w = _geo_row(x[idx], q[idx], nref[vi[idx], ui[idx]], z[idx], z_min, sim3)
    # ties and the bound on what their other outcomes change
    tie = valid & ((ur != ua) | (vr != va) | near | (np.abs(x[..., 2]) < TIE_X))
    dim = 7 if sim3 else 6
    tie_H, tie_g, tie_E = 0.0, np.zeros(dim), 0.0
    tix = np.nonzero(tie)
    if tix[0].size:
        rows_now = np.zeros((tix[0].size, dim, dim)), np.zeros((tix[0].size, dim)), np.zeros(tix[0].size)
        sel = ok[tix]
        if sel.any():
            t2 = (tix[0][sel], tix[1][sel])
            Jt, rt, wt = _geo_row(x[t2], q[t2], nref[vi[t2], ui[t2]], z[t2], z_min, sim3)
            cH, cg, cE = _contrib(Jt, rt, wt)
            rows_now[0][sel], rows_now[1][sel], rows_now[2][sel] = cH, cg, cE
        dH = np.linalg.norm(rows_now[0], axis=(1, 2))  # the "no row" outcome
        dg = np.abs(rows_now[1])
        dE = np.abs(rows_now[2])
        for uu, vv in ((ua, vr), (ur, va), (ua, va)):
            okc, nearc, uic, vic, qc = assoc(uu, vv)
            cand = (okc | nearc)[tix]
            if not cand.any():
                continue
            t2 = (tix[0][cand], tix[1][cand])
            Jc, rc, wc = _geo_row(x[t2], qc[t2], nref[vic[t2], uic[t2]], z[t2], z_min, sim3)
            cH, cg, cE = _contrib(Jc, rc, wc)
            dH[cand] = np.maximum(dH[cand], np.linalg.norm(cH - rows_now[0][cand], axis=(1, 2)))
            dg[cand] = np.maximum(dg[cand], np.abs(cg - rows_now[1][cand]))
            dE[cand] = np.maximum(dE[cand], np.abs(cE - rows_now[2][cand]))
        tie_H, tie_g, tie_E = float(dH.sum()), dg.sum(0), float(dE.sum())
    return Rows(J, r, w, J.shape[0], 0, int(tix[0].size), tie_H, tie_g, tie_E,
                np.stack(idx, -1), np.stack([vi[idx], ui[idx]], -1))


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
    from the render camera frame to the keyframe camera frame. A row exists where the
    point projects into [1, W - 2) x [1, H - 2) of the keyframe (the bilinear taps of the
    central-difference gradient stay inside) and |r| <= thr."""
    z = level.d64
    p = _backproject64(z, level.K)
    x = p @ dT[:3, :3].T + dT[:3, 3]
    y = x @ T_rs[:3, :3].T + T_rs[:3, 3]
    Hk, Wk = kf_I.shape
    valid = z > 0
    with np.errstate(divide="ignore", invalid="ignore"):
        zpos = y[..., 2] > 0
        uk = np.where(zpos, K_kf.fx * y[..., 0] / y[..., 2] + K_kf.cx, -1e9)
        vk = np.where(zpos, K_kf.fy * y[..., 1] / y[..., 2] + K_kf.cy, -1e9)
    inb = valid & zpos & (uk >= 1) & (vk >= 1) & (uk < Wk - 2) & (vk < Hk - 2)
    tie_b = valid & ((np.abs(uk - 1) < TIE_PX) | (np.abs(vk - 1) < TIE_PX) | (np.abs(uk - (Wk - 2)) < TIE_PX)
                     | (np.abs(vk - (Hk - 2)) < TIE_PX) | (np.abs(y[..., 2]) < TIE_X))
    gx, gy = grad_image(kf_I)
    # sample every pixel that is inside or a bound tie (clamped so the taps exist)
    cand = inb | tie_b
    idx = np.nonzero(cand)
    us = np.clip(uk[idx], 1.0, Wk - 2 - 1e-9)
    vs = np.clip(vk[idx], 1.0, Hk - 2 - 1e-9)
    Ik = bilinear(kf_I, us, vs)
    gxs = bilinear(gx, us, vs)
    gys = bilinear(gy, us, vs)
    r = level.I[idx] - Ik
    tie_r = np.abs(np.abs(r) - thr) < 1e-6 + TIE_PX * np.hypot(gxs, gys)
    keep_all = inb[idx] & (np.abs(r) <= thr)
    tie_all = tie_b[idx] | tie_r

    def rows(sel):
        yy, xx, rr, gxx, gyy = y[idx][sel], x[idx][sel], r[sel], gxs[sel], gys[sel]
        zz = z[idx][sel]
        X, Y, Z = yy[:, 0], yy[:, 1], yy[:, 2]
        # d(pi)/dy in pixels, rows (u, v)
        dpi = np.zeros((yy.shape[0], 2, 3))
        dpi[:, 0, 0] = K_kf.fx / Z
        dpi[:, 0, 2] = -K_kf.fx * X / Z ** 2
        dpi[:, 1, 1] = K_kf.fy / Z
        dpi[:, 1, 2] = -K_kf.fy * Y / Z ** 2
        gI = np.stack([gxx, gyy], axis=-1)                      # N x 2
        a = -np.einsum("ni,nij->nj", gI, dpi) @ T_rs[:3, :3]    # N x 3  (d r / d x in render frame)
        cols = [a, np.cross(xx, a)]                              # a . (-x^ e_k) = (x x a)_k
        if sim3:
            cols.append(np.einsum("ij,ij->i", a, xx)[:, None])
        return np.concatenate(cols, axis=1), rr, lam / (zz + (1.0 - z_min)) ** 2

    J, rr, w = rows(keep_all)
    dim = 7 if sim3 else 6
    tie_H, tie_g, tie_E = 0.0, np.zeros(dim), 0.0
    if tie_all.any():
        Jt, rt, wt = rows(tie_all)
        cH, cg, cE = _contrib(Jt, rt, wt)
        tie_H, tie_g, tie_E = float(np.linalg.norm(cH, axis=(1, 2)).sum()), np.abs(cg).sum(0), float(np.abs(cE).sum())
    pix = np.stack([idx[0][keep_all], idx[1][keep_all]], -1)
    return Rows(J, rr, w, 0, J.shape[0], int(tie_all.sum()), tie_H, tie_g, tie_E, pix, None)


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


def tie_bounds(rows: list[Rows]):
    """(tie pixels, bound on |dH|_F, bound on |dg| per component, bound on |dE|) of the rows' ties."""
    g = None
    for x in rows:
        if x.tie_g is not None:
            g = x.tie_g.copy() if g is None else g + x.tie_g
    return (sum(x.n_tie for x in rows), sum(x.tie_H for x in rows), g, sum(x.tie_E for x in rows))


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
