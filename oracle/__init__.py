"""FP64 CPU oracle of the DTSDF render + ICP hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or execute anything in this package.
It shares no code, headers, tables or constants with the CUDA library and never
imports it; the two meet only through the seeded inputs of ``scenes``.

* ``dtsdf_oracle.c`` (plain C, double precision): preprocessing, block
  allocation, voxel-projection fusion and ray-cast rendering (Sec. 3, 4, 7), and
  the view-dependent combined TSDF with its regular ray-cast (Sec. 4, Sec. 7).
* ``icp.py`` (numpy, double precision): pyramid, projective association,
  point-to-plane residuals and Jacobians in SE(3) and Sim(3), photometric
  frame-to-keyframe rows, normal equations, Cholesky solve and the exponential
  map (Sec. 5, 5.2, 5.3, 6).

Every value and every decision is computed in double precision. A decision whose
quantity lies within a stated margin of its threshold (the difference a single-
precision evaluation of the same quantity can make) is recorded as a tie: per pixel
(preprocess), per allocated (block, D) key (alloc_tie), per voxel (brick_ties) and per
ICP row (icp.Rows.tie). Comparisons with another implementation accept a difference
only on the oracle's ties, and report how many there were.

Parity status per function is listed in ``PARITY`` below. Every entry is pinned by
a test under ``tests/`` against closed forms, brute force, library routines or
invariants; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PARITY = {
    "w_dir": "pinned: closed-form values, partition of unity (tests/test_oracle_weights.py)",
    "preprocess": "pinned: exact plane normals, filter counts by brute force (tests/test_oracle_fusion.py)",
    "segment_blocks": "pinned: dense sampling of the segment and an independent half-open slab test "
                      "(tests/test_oracle_alloc.py)",
    "integrate": "pinned: per-voxel closed form on planes, running-average identity (tests/test_oracle_fusion.py)",
    "render": "pinned: analytic plane, sphere bound, thin-sheet lemma (tests/test_oracle_render.py)",
    "combine": "pinned: one direction's values kept, identical directions kept, hand-evaluated weights, analytic "
               "plane render (tests/test_oracle_combined.py)",
    "render_freespace": "pinned: analytic plane, thin-plate lemma, sphere bound, agreement with the direct render "
                        "(tests/test_oracle_freespace.py)",
    "filters": "pinned: constant / ramp / step invariants, scipy Gaussian correlation without range term, plane "
               "normals, MAE closed form (tests/test_oracle_filters.py)",
    "recycle": "pinned: brute-force criterion on every brick, fusion after recycling equal to fusion of a map "
               "that never held the removed bricks (tests/test_oracle_recycle.py)",
    "icp": "pinned: finite differences, exact recovery of known SE(3)/Sim(3) (tests/test_oracle_icp.py)",
    "exp": "pinned: Rodrigues closed form, group identities (tests/test_oracle_icp.py)",
}


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "dtsdf_oracle.c")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P, F, I, D = ctypes.c_void_p, ctypes.c_float, ctypes.c_int, ctypes.c_double
            L.om_create.argtypes = [F, F, F, F, F, F, F, F, I, I, P, I]
            L.om_create.restype = P
            L.om_free.argtypes = [P]
            L.om_num_bricks.argtypes = [P]
            L.om_num_bricks.restype = ctypes.c_int64
            L.om_bricks.argtypes = [P, P]
            L.om_brick_data.argtypes = [P, I, I, I, I, P]
            L.om_brick_data.restype = I
            L.om_brick_ties.argtypes = [P, I, I, I, I, P]
            L.om_brick_ties.restype = I
            L.om_alloc_tie.argtypes = [P, I, I, I, I]
            L.om_alloc_tie.restype = I
            L.om_export.argtypes = [P, ctypes.c_long, ctypes.c_long, P, P, P]
            L.om_export.restype = ctypes.c_long
            L.om_preprocess.argtypes = [P, I, I, F, F, F, F, F, F, F, P, P, P, P, P, P]
            L.om_preprocess.restype = I
            L.om_segment_blocks.argtypes = [P, P, D, P, P, P, I]
            L.om_segment_blocks.restype = I
            L.om_w_dir.argtypes = [D, D]
            L.om_w_dir.restype = D
            L.om_integrate.argtypes = [P, P, P, I, I, F, F, F, F, P]
            L.om_integrate.restype = I
            L.om_eval.argtypes = [P, P, P, P]
            L.om_eval.restype = I
            L.om_render.argtypes = [P, P, I, I, F, F, F, F, P, ctypes.c_long, P, P, P, P]
            L.om_render.restype = I
            L.om_combine.argtypes = [P, P]
            L.om_combine.restype = I
            L.om_render_combined.argtypes = [P, P, I, I, F, F, F, F, P, ctypes.c_long, P, P, P, P]
            L.om_render_combined.restype = I
            L.om_comb_voxel.argtypes = [P, I, I, I, P, P]
            L.om_comb_voxel.restype = I
            L.om_set_brick.argtypes = [P, I, I, I, I, P]
            L.om_set_brick.restype = I
            L.om_render_freespace.argtypes = [P, P, I, I, F, F, F, F, P, ctypes.c_long, P, P]
            L.om_render_freespace.restype = I
            L.om_render_count.argtypes = [P, P, I, I, F, F, F, F, P, ctypes.c_long, P]
            L.om_render_count.restype = I
            L.om_threads.argtypes = [I]
            L.om_threads.restype = I
            L.om_recycle.argtypes = [P, D]
            L.om_recycle.restype = ctypes.c_int64
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def w_dir(cos_angle: float, theta: float) -> float:
    """Eq. direction_weight (as read: clamp((theta - acos<n,v>) / (2 theta - pi/2), 0, 1))."""
    return _load().om_w_dir(float(cos_angle), float(theta))


def threads(n: int = 0) -> int:
    """Set the oracle's OpenMP thread count (n > 0) and return the count its loops use."""
    return int(_load().om_threads(int(n)))


def preprocess(depth: np.ndarray, K, z_min: float, z_max: float, delta_sup: float) -> dict:
    """Depth outlier filter and cross-product normals (Sec. 7), in double precision.
    ok / nok: kept pixel / pixel with a normal; tie: the normal's orientation toward the
    camera is within the tie margin; z: kept input depth; P, n: camera point and normal."""
    L = _load()
    d = np.ascontiguousarray(depth, np.float32)
    H, W = d.shape
    out = dict(ok=np.zeros((H, W), np.uint8), nok=np.zeros((H, W), np.uint8), tie=np.zeros((H, W), np.uint8),
               z=np.zeros((H, W), np.float32), P=np.zeros((H, W, 3), np.float64),
               n=np.zeros((H, W, 3), np.float64))
    rc = L.om_preprocess(_p(d), W, H, K.fx, K.fy, K.cx, K.cy, z_min, z_max, delta_sup,
                         _p(out["ok"]), _p(out["nok"]), _p(out["tie"]), _p(out["z"]), _p(out["P"]), _p(out["n"]))
    assert rc == 0
    return out


def segment_blocks(a, b, block_size: float, origin=(0.0, 0.0, 0.0)):
    """Blocks whose closed cube segment a-b meets (exact slab test, Sec. 7 allocation):
    (cells n x 3, met n bool, tie n bool); a cell is listed when it is met or a tie."""
    L = _load()
    A = np.ascontiguousarray(a, np.float64)
    B = np.ascontiguousarray(b, np.float64)
    O = np.ascontiguousarray(origin, np.float64)
    cells = np.zeros((256, 3), np.int32)
    flags = np.zeros(256, np.uint8)
    n = min(L.om_segment_blocks(_p(A), _p(B), float(block_size), _p(O), _p(cells), _p(flags), 256), 256)
    return cells[:n].copy(), (flags[:n] & 1) > 0, (flags[:n] & 2) > 0


class Params:
    """Map parameters (nominal single-precision values, as the library takes them)."""

    def __init__(self, voxel_size=0.005, truncation=0.02, theta=3 * np.pi / 8, w_max=255.0, w_carve=0.1,
                 z_min=0.1, z_max=6.0, delta_sup=None, carve_radius=2, dense_dim=0, origin=(0.0, 0.0, 0.0),
                 color=True):
        self.voxel_size = voxel_size
        self.truncation = truncation
        self.theta = theta
        self.w_max = w_max
        self.w_carve = w_carve
        self.z_min = z_min
        self.z_max = z_max
        self.delta_sup = truncation / 2 if delta_sup is None else delta_sup
        self.carve_radius = carve_radius
        self.dense_dim = dense_dim
        self.origin = tuple(origin)
        self.color = color


class OracleMap:
    """Directional TSDF in double precision: (block, D) hash of 8^3 bricks (Sec. 7)."""

    def __init__(self, params: Params):
        self.params = params
        L = _load()
        o = np.asarray(params.origin, np.float32)
        self._h = L.om_create(params.voxel_size, params.truncation, params.theta, params.w_max, params.w_carve,
                              params.z_min, params.z_max, params.delta_sup, params.carve_radius,
                              params.dense_dim, _p(o), int(params.color))
        if not self._h:
            raise MemoryError("oracle map creation failed")
        self._L = L

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.om_free(self._h)
            self._h = None

    def integrate(self, depth, rgb, K, T_wc):
        d = np.ascontiguousarray(depth, np.float32)
        c = None if rgb is None else np.ascontiguousarray(rgb, np.uint8)
        T = np.ascontiguousarray(T_wc, np.float64)
        rc = self._L.om_integrate(self._h, _p(d), _p(c), d.shape[1], d.shape[0], K.fx, K.fy, K.cx, K.cy, _p(T))
        if rc != 0:
            raise MemoryError("oracle integrate failed")

    def recycle(self, free_sdf: float = 0.75) -> int:
        """Remove the bricks whose weighted voxels all have sdf >= free_sdf (Sec. 3 recycling)."""
        return int(self._L.om_recycle(self._h, float(np.float32(free_sdf))))

    def num_bricks(self) -> int:
        return int(self._L.om_num_bricks(self._h))

    def bricks(self) -> np.ndarray:
        """n x 5 int32: bx, by, bz, D, frame of first allocation."""
        n = self.num_bricks()
        out = np.zeros((n, 5), np.int32)
        if n:
            self._L.om_bricks(self._h, _p(out))
        return out

    def brick(self, bx, by, bz, D) -> np.ndarray | None:
        """512 x 6 doubles (sdf, w, r, g, b, wc), voxel index i + 8 j + 64 k."""
        out = np.zeros((512, 6), np.float64)
        rc = self._L.om_brick_data(self._h, int(bx), int(by), int(bz), int(D), _p(out))
        return None if rc != 0 else out

    def brick_ties(self, bx, by, bz, D) -> np.ndarray | None:
        """512 tie flags (bit 0: sdf and weight, bit 1: colour) of a brick's voxels."""
        out = np.zeros(512, np.uint8)
        rc = self._L.om_brick_ties(self._h, int(bx), int(by), int(bz), int(D), _p(out))
        return None if rc != 0 else out

    def export(self, start: int = 0, count: int | None = None):
        """Bricks [start, start + count) in map order: (coords int32 [n, 4], voxels float64
        [n, 512, 6] as brick(), ties uint8 [n, 512] as brick_ties())."""
        nb = self.num_bricks()
        count = nb - start if count is None else max(0, min(count, nb - start))
        coords = np.zeros((count, 4), np.int32)
        vox = np.zeros((count, 512, 6), np.float64)
        ties = np.zeros((count, 512), np.uint8)
        if count:
            self._L.om_export(self._h, int(start), int(count), _p(coords), _p(vox), _p(ties))
        return coords, vox, ties

    def alloc_tie(self, bx, by, bz, D) -> int:
        """First frame whose allocation of (bx, by, bz, D) was a tie, -1 if none was."""
        return int(self._L.om_alloc_tie(self._h, int(bx), int(by), int(bz), int(D)))

    def set_brick(self, bx, by, bz, D, vox):
        """Write a brick (512 x 6: sdf, w, r, g, b, wc), allocating it if needed (tests)."""
        v = np.ascontiguousarray(vox, np.float64).reshape(512, 6)
        if self._L.om_set_brick(self._h, int(bx), int(by), int(bz), int(D), _p(v)) != 0:
            raise MemoryError("oracle set_brick failed")

    def eval(self, x, r):
        info = np.zeros(9, np.float64)
        ok = self._L.om_eval(self._h, _p(np.ascontiguousarray(x, np.float64)),
                             _p(np.ascontiguousarray(r, np.float64)), _p(info))
        return bool(ok), info

    def combine(self, centre):
        """View-dependent combined TSDF of every allocated block for the camera centre (Sec. 4, Sec. 7)."""
        if self._L.om_combine(self._h, _p(np.ascontiguousarray(centre, np.float64))) != 0:
            raise MemoryError("oracle combine failed")

    def comb_voxel(self, x, y, z, centre):
        """(defined, phi, rgb, colour ok) of the combined value of voxel (x, y, z)."""
        info = np.zeros(5, np.float64)
        ok = self._L.om_comb_voxel(self._h, int(x), int(y), int(z), _p(np.ascontiguousarray(centre, np.float64)),
                                   _p(info))
        return bool(ok), info[0], info[1:4], bool(info[4])

    def render_combined(self, K, T_wc, pixels: np.ndarray | None = None):
        """Ray-cast of the combined TSDF of the last combine(); outputs as render()."""
        return self._render(self._L.om_render_combined, K, T_wc, pixels)

    def render(self, K, T_wc, pixels: np.ndarray | None = None):
        """Ray-cast depth (0 = miss), camera-frame normals, colour, colour validity."""
        return self._render(self._L.om_render, K, T_wc, pixels)

    def render_count(self, K, T_wc, pixels: np.ndarray | None = None) -> dict:
        """Distinct bricks read by the march, block cells whose hash entry it reads, colour voxels
        entering the outputs, and hits, for a render of the pixels (all if None)."""
        T = np.ascontiguousarray(T_wc, np.float64)
        pix = None if pixels is None else np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
        n = K.width * K.height if pix is None else pix.shape[0]
        c = np.zeros(4, np.int64)
        if self._L.om_render_count(self._h, _p(T), K.width, K.height, K.fx, K.fy, K.cx, K.cy, _p(pix), n, _p(c)) != 0:
            raise MemoryError("oracle render_count failed")
        return dict(bricks=int(c[0]), cells=int(c[1]), colour_voxels=int(c[2]), hits=int(c[3]))

    def render_freespace(self, K, T_wc, pixels: np.ndarray | None = None):
        """Ray-cast with the free-space combination of Alg. 1: depth (0 = miss), camera-frame
        normals (no colour)."""
        T = np.ascontiguousarray(T_wc, np.float64)
        if pixels is None:
            n = K.width * K.height
            pix = None
        else:
            pix = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
            n = pix.shape[0]
        depth = np.zeros(n, np.float64)
        normal = np.zeros((n, 3), np.float64)
        self._L.om_render_freespace(self._h, _p(T), K.width, K.height, K.fx, K.fy, K.cx, K.cy,
                                    None if pix is None else _p(pix), n, _p(depth), _p(normal))
        if pixels is None:
            return depth.reshape(K.height, K.width), normal.reshape(K.height, K.width, 3)
        return depth, normal

    def _render(self, fn, K, T_wc, pixels):
        T = np.ascontiguousarray(T_wc, np.float64)
        if pixels is None:
            n = K.width * K.height
            pix = None
        else:
            pix = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
            n = pix.shape[0]
        depth = np.zeros(n, np.float64)
        normal = np.zeros((n, 3), np.float64)
        color = np.zeros((n, 3), np.float64)
        cok = np.zeros(n, np.uint8)
        rc = fn(self._h, _p(T), K.width, K.height, K.fx, K.fy, K.cx, K.cy, _p(pix), n, _p(depth), _p(normal),
                _p(color), _p(cok))
        if rc != 0:
            raise RuntimeError("oracle render failed (combined: call combine() first)")
        if pixels is None:
            return (depth.reshape(K.height, K.width), normal.reshape(K.height, K.width, 3),
                    color.reshape(K.height, K.width, 3), cok.reshape(K.height, K.width))
        return depth, normal, color, cok
