"""FP64 oracle of the bilateral input filters and the post-fusion error (test infrastructure
only: tests/, smoke() and bench.py's CPU baseline use it; the product never imports it).

Passages followed:
  * Sec. 8 settings: bilateral depth filter sigma_d = 5.0, sigma_r = 0.025, radius 5; bilateral
    normal filter sigma_d = 2.5, sigma_r = 5.0, radius 5. The paper gives no formula: these are
    the usual bilateral filters - a normalised sum over the (2r+1)^2 window of the valid pixels,
    weighted by a Gaussian of the pixel distance (sigma_d, pixels) times a Gaussian of the value
    difference (depth: metres; normals: the angle between them in degrees).
  * Sec. 7: normals are the cross product of the central differences of the back-projected
    neighbours in x and y, turned toward the camera, present where the pixel and its four
    neighbours are.
  * Sec. 8.2: the post-fusion error of a frame is the mean absolute difference between the depth
    rendered at its estimated pose and its input depth, over the pixels where both exist.
"""
from __future__ import annotations

import numpy as np


def _shift(a: np.ndarray, dv: int, du: int, fill=0.0) -> np.ndarray:
    """out[v, u] = a[v + dv, u + du] where inside the image, else fill."""
    H, W = a.shape[:2]
    out = np.full_like(a, fill)
    sv = slice(max(dv, 0), H + min(dv, 0))
    tv = slice(max(-dv, 0), H + min(-dv, 0))
    su = slice(max(du, 0), W + min(du, 0))
    tu = slice(max(-du, 0), W + min(-du, 0))
    out[tv, tu] = a[sv, su]
    return out


def bilateral_depth(z: np.ndarray, radius: int, sigma_d: float, sigma_r: float) -> np.ndarray:
    """Bilateral depth filter over the valid (> 0) pixels of z; invalid pixels stay 0."""
    z = np.asarray(z, np.float64)
    valid = z > 0
    num = np.zeros_like(z)
    den = np.zeros_like(z)
    for dv in range(-radius, radius + 1):
        for du in range(-radius, radius + 1):
            zj = _shift(z, dv, du)
            ok = valid & (zj > 0)
            w = np.exp(-(du * du + dv * dv) / (2.0 * sigma_d ** 2)) * np.exp(-((zj - z) ** 2) / (2.0 * sigma_r ** 2))
            num += np.where(ok, w * zj, 0.0)
            den += np.where(ok, w, 0.0)
    return np.where(valid, num / np.where(valid, den, 1.0), 0.0)


def backproject(z: np.ndarray, K) -> np.ndarray:
    """Eq. reprojection: (z (u - cx)/fx, z (v - cy)/fy, z)."""
    H, W = z.shape
    u = np.arange(W, dtype=np.float64)[None, :]
    v = np.arange(H, dtype=np.float64)[:, None]
    return np.stack([z * (u - K.cx) / K.fx, z * (v - K.cy) / K.fy, np.asarray(z, np.float64)], axis=-1)


def normals(P: np.ndarray, valid: np.ndarray):
    """Sec. 7 normals of the point image P [H, W, 3] (valid: [H, W] bool). Returns (n, has_n)."""
    H, W = valid.shape
    n = np.zeros((H, W, 3))
    has = np.zeros((H, W), bool)
    has[1:-1, 1:-1] = (valid[1:-1, 1:-1] & valid[1:-1, :-2] & valid[1:-1, 2:] & valid[:-2, 1:-1]
                       & valid[2:, 1:-1])
    dx = P[1:-1, 2:] - P[1:-1, :-2]
    dy = P[2:, 1:-1] - P[:-2, 1:-1]
    c = np.cross(dx, dy)
    ln = np.linalg.norm(c, axis=-1, keepdims=True)
    c = c / np.where(ln > 0, ln, 1.0)
    flip = np.sum(c * P[1:-1, 1:-1], axis=-1) > 0
    c[flip] = -c[flip]
    n[1:-1, 1:-1] = c
    has[1:-1, 1:-1] &= ln[..., 0] > 0
    n[~has] = 0.0
    return n, has


def bilateral_normals(n: np.ndarray, has: np.ndarray, radius: int, sigma_d: float, sigma_r_deg: float) -> np.ndarray:
    """Bilateral normal filter: normalised weighted sum of the window's normals, range term on the
    angle between the normals in degrees. Pixels without a normal stay 0."""
    acc = np.zeros_like(n)
    for dv in range(-radius, radius + 1):
        for du in range(-radius, radius + 1):
            nj = _shift(n, dv, du)
            ok = has & _shift(has.astype(np.float64), dv, du).astype(bool)
            ang = np.degrees(np.arccos(np.clip(np.sum(n * nj, axis=-1), -1.0, 1.0)))
            w = np.exp(-(du * du + dv * dv) / (2.0 * sigma_d ** 2)) * np.exp(-(ang ** 2) / (2.0 * sigma_r_deg ** 2))
            acc += np.where(ok, w, 0.0)[..., None] * nj
    ln = np.linalg.norm(acc, axis=-1, keepdims=True)
    out = acc / np.where(ln > 0, ln, 1.0)
    out[~has] = 0.0
    return out


def depth_mae(rendered: np.ndarray, measured: np.ndarray):
    """Sec. 8.2 post-fusion error of one frame: (sum |rendered - measured|, count) over the pixels
    where both depths are positive."""
    a = np.asarray(rendered, np.float64)
    b = np.asarray(measured, np.float64)
    both = (a > 0) & (b > 0)
    return float(np.sum(np.abs(a - b)[both])), int(np.count_nonzero(both))
