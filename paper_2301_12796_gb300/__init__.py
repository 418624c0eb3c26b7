"""Python binding of libdtsdf (the C ABI declared in include/dtsdf.h).

Argument marshalling only: every step of fusion, rendering and ICP runs in the
library's CUDA kernels. PyTorch tensors provide device memory and streams; their
data pointers are passed straight through. There is no CPU fallback: if the
shared library is missing or cannot be loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdtsdf.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_OOM, ERR_MAP_FULL, ERR_CUDA, ERR_DEGENERATE, ERR_TIMEOUT = range(7)
STORE_FP32, STORE_FP16 = 0, 1
_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "MAP_FULL", 4: "CUDA", 5: "DEGENERATE", 6: "TIMEOUT"}

c_float, c_int32, c_uint32, c_int64, c_double, c_void_p = (ctypes.c_float, ctypes.c_int32, ctypes.c_uint32,
                                                          ctypes.c_int64, ctypes.c_double, ctypes.c_void_p)


class Params(ctypes.Structure):
    _fields_ = [("voxel_size", c_float), ("truncation", c_float), ("theta", c_float), ("w_max", c_float),
                ("w_carve", c_float), ("z_min", c_float), ("z_max", c_float), ("delta_sup", c_float),
                ("carve_radius", c_int32), ("dense_dim", c_int32), ("dense_origin", c_float * 3),
                ("max_blocks", c_uint32), ("storage", c_int32), ("color", c_int32)]


class Intrinsics(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float)]


class Frame(ctypes.Structure):
    _fields_ = [("depth", c_void_p), ("rgb", c_void_p), ("K", Intrinsics)]


class RenderOut(ctypes.Structure):
    _fields_ = [("depth", c_void_p), ("normals", c_void_p), ("color", c_void_p)]


class RenderOpts(ctypes.Structure):
    _fields_ = [("ctas", c_int32), ("refill", c_int32), ("tile_w", c_int32)]


class FilterOpts(ctypes.Structure):
    _fields_ = [("depth_radius", c_int32), ("depth_sigma_d", c_float), ("depth_sigma_r", c_float),
                ("normal_radius", c_int32), ("normal_sigma_d", c_float), ("normal_sigma_r", c_float)]


def filter_opts(depth=True, normals=True, depth_radius=5, depth_sigma_d=5.0, depth_sigma_r=0.025, normal_radius=5,
                normal_sigma_d=2.5, normal_sigma_r=5.0) -> FilterOpts:
    """Bilateral input filters with the Sec. 8 settings by default; a filter that is not wanted
    gets radius 0."""
    return FilterOpts(depth_radius if depth else 0, depth_sigma_d, depth_sigma_r, normal_radius if normals else 0,
                      normal_sigma_d, normal_sigma_r)


class IcpProblem(ctypes.Structure):
    _fields_ = [("icp", c_void_p), ("ref", RenderOut), ("K_ref", Intrinsics), ("T_rel_dev", c_void_p),
                ("stats_dev", c_void_p), ("sim3", c_int32)]


class BatchShape(ctypes.Structure):
    _fields_ = [("cluster", c_int32), ("threads", c_int32)]


class RenderJob(ctypes.Structure):
    _fields_ = [("K", Intrinsics), ("T_wc_dev", c_void_p), ("out", RenderOut)]


class MapStats(ctypes.Structure):
    _fields_ = [("bricks", c_int64), ("blocks", c_int64), ("bricks_per_dir", c_int64 * 6), ("capacity", c_int64),
                ("error_flags", c_uint32), ("frames", c_int32)]


class IcpOpts(ctypes.Structure):
    _fields_ = [("levels", c_int32), ("iters", c_int32 * 4), ("eps", c_float * 4), ("photo_thr", c_float * 4),
                ("lambda_", c_float), ("z_min", c_float), ("stop_norm", c_double), ("min_rows", c_int32),
                ("kahan", c_int32), ("lm", c_int32)]


class IcpStats(ctypes.Structure):
    _fields_ = [("H", c_double * 49), ("g", c_double * 7), ("xi", c_double * 7), ("error", c_double),
                ("rows", c_int64), ("rows_photo", c_int64), ("step_norm", c_double), ("dim", c_int32),
                ("status", c_int32), ("converged", c_int32), ("iterations", c_int32)]

    def H_matrix(self) -> np.ndarray:
        d = self.dim
        return np.array(self.H[:], np.float64).reshape(7, 7)[:d, :d].copy()

    def g_vector(self) -> np.ndarray:
        return np.array(self.g[: self.dim], np.float64)


class ServerParams(ctypes.Structure):
    _fields_ = [("hbm_budget", c_int64), ("max_inflight", c_int32), ("max_batch", c_int32), ("streams", c_int32),
                ("max_width", c_int32), ("max_height", c_int32), ("z_min", c_float), ("z_max", c_float),
                ("delta_sup", c_float), ("opts", IcpOpts), ("shape", BatchShape)]


class Request(ctypes.Structure):
    _fields_ = [("map", c_int32), ("sim3", c_int32), ("K", Intrinsics), ("depth", c_void_p),
                ("T_prior", c_double * 16), ("tag", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("seq", ctypes.c_uint64), ("status", c_int32), ("batch_size", c_int32),
                ("T_rel", c_double * 16), ("T_wc", c_double * 16), ("stats", IcpStats), ("t_submit", c_double),
                ("t_admit", c_double), ("t_done", c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, c_int64) for n in ("submitted", "admitted", "completed", "batches", "pending", "inflight",
                                       "peak_inflight", "bytes_in_use", "peak_bytes")]


# exported symbols and their signatures (every function include/dtsdf.h declares)
P = c_void_p
SIGNATURES = {
    "dtsdf_create": ([ctypes.POINTER(Params), P, ctypes.POINTER(P)], c_int32),
    "dtsdf_destroy": ([P], c_int32),
    "dtsdf_integrate": ([P, ctypes.POINTER(Frame), P, P], c_int32),
    "dtsdf_integrate_dev": ([P, ctypes.POINTER(Frame), P, P], c_int32),
    "dtsdf_render": ([P, ctypes.POINTER(Intrinsics), P, ctypes.POINTER(RenderOut), P], c_int32),
    "dtsdf_render_dev": ([P, ctypes.POINTER(Intrinsics), P, ctypes.POINTER(RenderOut), P], c_int32),
    "dtsdf_render_combined": ([P, ctypes.POINTER(Intrinsics), P, ctypes.POINTER(RenderOut), P], c_int32),
    "dtsdf_render_combined_dev": ([P, ctypes.POINTER(Intrinsics), P, ctypes.POINTER(RenderOut), P], c_int32),
    "dtsdf_combined_reset": ([P], c_int32),
    "dtsdf_combine": ([P, ctypes.POINTER(Intrinsics), P, c_int32, P], c_int32),
    "dtsdf_combine_dev": ([P, ctypes.POINTER(Intrinsics), P, c_int32, P], c_int32),
    "dtsdf_combined_blocks": ([P, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64), P], c_int32),
    "dtsdf_live_allocations": ([], ctypes.c_int64),
    "dtsdf_set_render_opts": ([P, ctypes.POINTER(RenderOpts)], c_int32),
    "dtsdf_render_tune": ([P, ctypes.POINTER(Intrinsics), P, ctypes.POINTER(RenderOut), ctypes.POINTER(RenderOpts),
                           ctypes.POINTER(ctypes.c_float), P], c_int32),
    "dtsdf_render_touched": ([P, ctypes.POINTER(Intrinsics), P, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                              P, P], c_int32),
    "dtsdf_pose_compose": ([P, c_int32, P, P, P], c_int32),
    "dtsdf_map_stats": ([P, ctypes.POINTER(MapStats), P], c_int32),
    "dtsdf_map_export": ([P, P, P, c_int64, ctypes.POINTER(c_int64), P], c_int32),
    "dtsdf_map_import": ([P, P, P, c_int64, P], c_int32),
    "dtsdf_icp_create": ([c_int32, c_int32, c_int32, ctypes.POINTER(P)], c_int32),
    "dtsdf_icp_destroy": ([P], c_int32),
    "dtsdf_icp_set_frame": ([P, ctypes.POINTER(Frame), c_float, c_float, c_float, P], c_int32),
    "dtsdf_icp_set_keyframe": ([P, ctypes.POINTER(Frame), P], c_int32),
    "dtsdf_icp_step": ([P, ctypes.POINTER(RenderOut), ctypes.POINTER(Intrinsics), c_int32, P, P,
                        ctypes.POINTER(IcpOpts), ctypes.POINTER(IcpStats), P], c_int32),
    "dtsdf_icp_sim3_step": ([P, ctypes.POINTER(RenderOut), ctypes.POINTER(Intrinsics), c_int32, P, P,
                             ctypes.POINTER(IcpOpts), ctypes.POINTER(IcpStats), P], c_int32),
    "dtsdf_icp_solve": ([P, ctypes.POINTER(RenderOut), ctypes.POINTER(Intrinsics), c_int32, P, P,
                         ctypes.POINTER(IcpOpts), P, P], c_int32),
    "dtsdf_icp_step_noalloc": ([P, ctypes.POINTER(Intrinsics), ctypes.POINTER(RenderOut),
                                ctypes.POINTER(Intrinsics), c_int32, c_float, c_float, c_int32, c_double, P, P, P],
                               c_int32),
    "dtsdf_icp_batch": ([ctypes.POINTER(IcpProblem), c_int32, ctypes.POINTER(IcpOpts), ctypes.POINTER(BatchShape), P],
                        c_int32),
    "dtsdf_icp_batch_tune": ([ctypes.POINTER(IcpProblem), c_int32, ctypes.POINTER(IcpOpts),
                              ctypes.POINTER(BatchShape), ctypes.POINTER(ctypes.c_float), P], c_int32),
    "dtsdf_render_batch": ([P, ctypes.POINTER(RenderJob), c_int32, P], c_int32),
    "dtsdf_server_create": ([ctypes.POINTER(P), c_int32, ctypes.POINTER(ServerParams), ctypes.POINTER(P)], c_int32),
    "dtsdf_server_submit": ([P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)], c_int32),
    "dtsdf_server_poll": ([P, ctypes.POINTER(Result), c_int32, ctypes.POINTER(c_int32), c_int32], c_int32),
    "dtsdf_server_stats": ([P, ctypes.POINTER(ServerStats)], c_int32),
    "dtsdf_server_clock": ([P], c_double),
    "dtsdf_server_destroy": ([P], c_int32),
    "dtsdf_exp": ([c_int32, P, P], c_int32),
    "dtsdf_recycle": ([P, c_float, ctypes.POINTER(c_int64), P], c_int32),
    "dtsdf_render_freespace": ([P, ctypes.POINTER(Intrinsics), P, ctypes.POINTER(RenderOut), P], c_int32),
    "dtsdf_render_freespace_dev": ([P, ctypes.POINTER(Intrinsics), P, ctypes.POINTER(RenderOut), P], c_int32),
    "dtsdf_set_filters": ([P, ctypes.POINTER(FilterOpts)], c_int32),
    "dtsdf_icp_set_filters": ([P, ctypes.POINTER(FilterOpts)], c_int32),
    "dtsdf_preprocess": ([ctypes.POINTER(Frame), c_float, c_float, c_float, ctypes.POINTER(FilterOpts), P, P, P],
                         c_int32),
    "dtsdf_depth_mae": ([P, P, c_int64, P, P], c_int32),
    "dtsdf_scale_anchor": ([P, P, c_int64, c_int32, c_double, P], c_int32),
    "dtsdf_depth_scale": ([P, P, c_int64, c_float, P], c_int32),
    "dtsdf_last_error": ([], ctypes.c_char_p),
    "dtsdf_version": ([], ctypes.c_char_p),
}


class DtsdfError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libdtsdf.so (build it first with paper_2301_12796_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libdtsdf.so not built ({LIB_PATH}); run python -m paper_2301_12796_gb300.build")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def check(status: int, where: str):
    if status != OK:
        raise DtsdfError(status, where, lib().dtsdf_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def intrinsics(K) -> Intrinsics:
    return Intrinsics(int(K.width), int(K.height), float(K.fx), float(K.fy), float(K.cx), float(K.cy))


def pose_buf(T) -> ctypes.Array:
    a = np.ascontiguousarray(np.asarray(T, np.float64).reshape(16))
    return (c_double * 16)(*a.tolist())


def params(voxel_size=0.005, truncation=0.02, theta=3 * np.pi / 8, w_max=255.0, w_carve=0.1, z_min=0.1, z_max=6.0,
           delta_sup=None, carve_radius=2, dense_dim=0, origin=(0.0, 0.0, 0.0), max_blocks=1 << 16,
           storage=STORE_FP32, color=True) -> Params:
    return Params(voxel_size, truncation, theta, w_max, w_carve, z_min, z_max,
                  truncation / 2 if delta_sup is None else delta_sup, carve_radius, dense_dim,
                  (c_float * 3)(*origin), max_blocks, storage, int(color))


class Map:
    """A Directional TSDF in device memory (dtsdf_create / dtsdf_destroy)."""

    def __init__(self, p: Params, stream=None):
        self.params = p
        h = c_void_p()
        check(lib().dtsdf_create(ctypes.byref(p), _stream_ptr(stream), ctypes.byref(h)), "dtsdf_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dtsdf_destroy(self._h)
            self._h = None

    __del__ = close

    def integrate(self, depth, rgb, K, T_wc, stream=None):
        """depth: float32 CUDA tensor [H, W]; rgb: uint8 CUDA tensor [H, W, 3] or None."""
        f = Frame(depth.data_ptr(), None if rgb is None else rgb.data_ptr(), intrinsics(K))
        check(lib().dtsdf_integrate(self._h, ctypes.byref(f), pose_buf(T_wc), _stream_ptr(stream)),
              "dtsdf_integrate")

    def render(self, K, T_wc, depth, normals, color=None, stream=None):
        """depth [H, W] float32, normals [H, W, 4] float32, color [H, W, 4] float32 or None (CUDA tensors)."""
        out = RenderOut(depth.data_ptr(), normals.data_ptr(), None if color is None else color.data_ptr())
        Ki = intrinsics(K)
        check(lib().dtsdf_render(self._h, ctypes.byref(Ki), pose_buf(T_wc), ctypes.byref(out), _stream_ptr(stream)),
              "dtsdf_render")

    def integrate_dev(self, depth, rgb, K, T_dev, stream=None):
        """Fuse at the pose held by the float64 CUDA tensor T_dev [4, 4]."""
        f = Frame(depth.data_ptr(), None if rgb is None else rgb.data_ptr(), intrinsics(K))
        check(lib().dtsdf_integrate_dev(self._h, ctypes.byref(f), T_dev.data_ptr(), _stream_ptr(stream)),
              "dtsdf_integrate_dev")

    def render_dev(self, K, T_dev, depth, normals, color=None, stream=None):
        out = RenderOut(depth.data_ptr(), normals.data_ptr(), None if color is None else color.data_ptr())
        Ki = intrinsics(K)
        check(lib().dtsdf_render_dev(self._h, ctypes.byref(Ki), T_dev.data_ptr(), ctypes.byref(out),
                                     _stream_ptr(stream)), "dtsdf_render_dev")

    def render_combined(self, K, T_wc, depth, normals, color=None, stream=None):
        """Render from the view-dependent combined TSDF with conditional combination (host pose)."""
        out = RenderOut(depth.data_ptr(), normals.data_ptr(), None if color is None else color.data_ptr())
        Ki = intrinsics(K)
        check(lib().dtsdf_render_combined(self._h, ctypes.byref(Ki), pose_buf(T_wc), ctypes.byref(out),
                                          _stream_ptr(stream)), "dtsdf_render_combined")

    def render_combined_dev(self, K, T_dev, depth, normals, color=None, stream=None):
        """Same with the pose in the float64 CUDA tensor T_dev [4, 4]."""
        out = RenderOut(depth.data_ptr(), normals.data_ptr(), None if color is None else color.data_ptr())
        Ki = intrinsics(K)
        check(lib().dtsdf_render_combined_dev(self._h, ctypes.byref(Ki), T_dev.data_ptr(), ctypes.byref(out),
                                              _stream_ptr(stream)), "dtsdf_render_combined_dev")

    def combine(self, K, T_wc, force=False, stream=None):
        """The combination step alone (host pose); force recombines the whole padded frustum."""
        Ki = intrinsics(K)
        check(lib().dtsdf_combine(self._h, ctypes.byref(Ki), pose_buf(T_wc), int(bool(force)), _stream_ptr(stream)),
              "dtsdf_combine")

    def combine_dev(self, K, T_dev, force=False, stream=None):
        Ki = intrinsics(K)
        check(lib().dtsdf_combine_dev(self._h, ctypes.byref(Ki), T_dev.data_ptr(), int(bool(force)),
                                      _stream_ptr(stream)), "dtsdf_combine_dev")

    def combined_blocks(self, stream=None):
        """(blocks, bricks) of the current combination."""
        b, k = c_int64(), c_int64()
        check(lib().dtsdf_combined_blocks(self._h, ctypes.byref(b), ctypes.byref(k), _stream_ptr(stream)),
              "dtsdf_combined_blocks")
        return b.value, k.value

    def combined_reset(self):
        """The next combined render recombines the whole frustum at its pose."""
        check(lib().dtsdf_combined_reset(self._h), "dtsdf_combined_reset")

    def render_batch(self, jobs, stream=None):
        """Render several frames in one launch. jobs: list of (K, T_dev float64 [4, 4] CUDA tensor,
        depth [H, W], normals [H, W, 4], color [H, W, 4] or None)."""
        arr = (RenderJob * max(len(jobs), 1))()
        for i, (K, T_dev, depth, normals, color) in enumerate(jobs):
            arr[i] = RenderJob(intrinsics(K), T_dev.data_ptr(),
                               RenderOut(depth.data_ptr(), normals.data_ptr(), None if color is None else color.data_ptr()))
        check(lib().dtsdf_render_batch(self._h, arr, len(jobs), _stream_ptr(stream)), "dtsdf_render_batch")

    def render_freespace(self, K, T_wc, depth, normals, color=None, stream=None):
        """Render with the free-space combination of Alg. 1 (quality reference; no colour)."""
        out = RenderOut(depth.data_ptr(), normals.data_ptr(), None if color is None else color.data_ptr())
        Ki = intrinsics(K)
        check(lib().dtsdf_render_freespace(self._h, ctypes.byref(Ki), pose_buf(T_wc), ctypes.byref(out),
                                           _stream_ptr(stream)), "dtsdf_render_freespace")

    def render_freespace_dev(self, K, T_dev, depth, normals, color=None, stream=None):
        out = RenderOut(depth.data_ptr(), normals.data_ptr(), None if color is None else color.data_ptr())
        Ki = intrinsics(K)
        check(lib().dtsdf_render_freespace_dev(self._h, ctypes.byref(Ki), T_dev.data_ptr(), ctypes.byref(out),
                                               _stream_ptr(stream)), "dtsdf_render_freespace_dev")

    def set_filters(self, f: FilterOpts | None):
        """Bilateral input filters of this map's fusion (None: off)."""
        check(lib().dtsdf_set_filters(self._h, None if f is None else ctypes.byref(f)), "dtsdf_set_filters")

    def set_render_opts(self, ctas: int = 0, refill: int = 0, tile_w: int = 0):
        """Launch shape of this map's renders: persistent CTAs (0 = one resident wave), lanes per
        refill group (1, 2, 4, 8, 16, 32; 0 = 32) and the width of the 32-ray pixel tiles (1, 2, 4,
        8, 16, 32; 0 = 4). Every shape gives the same outputs."""
        o = RenderOpts(int(ctas), int(refill), int(tile_w))
        check(lib().dtsdf_set_render_opts(self._h, ctypes.byref(o)), "dtsdf_set_render_opts")

    def tune_render(self, K, T_wc, depth, normals, color=None, stream=None):
        """Time every render launch shape at T_wc, keep the fastest; returns ((ctas, refill,
        tile_w), ms)."""
        out = RenderOut(depth.data_ptr(), normals.data_ptr(), None if color is None else color.data_ptr())
        Ki = intrinsics(K)
        best = RenderOpts()
        ms = ctypes.c_float()
        check(lib().dtsdf_render_tune(self._h, ctypes.byref(Ki), pose_buf(T_wc), ctypes.byref(out), ctypes.byref(best),
                                      ctypes.byref(ms), _stream_ptr(stream)), "dtsdf_render_tune")
        return (best.ctas, best.refill, best.tile_w), ms.value

    def touched(self, K, T_wc, stream=None, counters=False):
        """(geometry bricks, colour bricks) read by one render at T_wc; with counters=True also
        a dict of per-frame totals (samples, full combinations, cells, allocated cells, hits)."""
        g, c = c_int64(), c_int64()
        ctr = (c_int64 * 8)()
        Ki = intrinsics(K)
        check(lib().dtsdf_render_touched(self._h, ctypes.byref(Ki), pose_buf(T_wc), ctypes.byref(g), ctypes.byref(c),
                                         ctr, _stream_ptr(stream)), "dtsdf_render_touched")
        if counters:
            names = ["samples", "full", "cells", "alloc_cells", "hits", "cell_jumps"]
            return g.value, c.value, {n: int(ctr[i]) for i, n in enumerate(names)}
        return g.value, c.value

    def stats(self, stream=None) -> MapStats:
        st = MapStats()
        check(lib().dtsdf_map_stats(self._h, ctypes.byref(st), _stream_ptr(stream)), "dtsdf_map_stats")
        return st

    def recycle(self, free_sdf: float = 0.75, stream=None) -> int:
        """Return the bricks whose weighted voxels are all >= free_sdf to the pool (dtsdf_recycle);
        returns how many were detached."""
        n = c_int64()
        check(lib().dtsdf_recycle(self._h, float(free_sdf), ctypes.byref(n), _stream_ptr(stream)), "dtsdf_recycle")
        return int(n.value)

    def export(self, stream=None):
        """(coords int32 [n, 4] = bx, by, bz, D; voxels float32 [n, 512, 6] = sdf, w, r, g, b, wc) of the
        live bricks (pool entries of recycled bricks are left out)."""
        n = c_int64()
        check(lib().dtsdf_map_export(self._h, None, None, 0, ctypes.byref(n), _stream_ptr(stream)), "export")
        coords = np.zeros((n.value, 4), np.int32)
        vox = np.zeros((n.value, 512, 6), np.float32)
        if n.value:
            check(lib().dtsdf_map_export(self._h, coords.ctypes.data_as(c_void_p), vox.ctypes.data_as(c_void_p),
                                         n.value, ctypes.byref(n), _stream_ptr(stream)), "export")
        live = coords[:, 3] >= 0
        if not live.all():
            coords, vox = coords[live], vox[live]
        return coords, vox


def _import(self, coords, voxels, stream=None):
    """Load bricks (coords int32 [n, 4], voxels float32 [n, 512, 6]) into the map."""
    c = np.ascontiguousarray(coords, np.int32)
    v = np.ascontiguousarray(voxels, np.float32)
    assert c.shape[0] == v.shape[0] and c.shape[1:] == (4,) and v.shape[1:] == (512, 6)
    check(lib().dtsdf_map_import(self._h, c.ctypes.data_as(c_void_p), v.ctypes.data_as(c_void_p), c.shape[0],
                                 _stream_ptr(stream)), "dtsdf_map_import")


Map.import_bricks = _import


def icp_opts(levels=3, iters=(10, 5, 4), eps=(0.005, 0.05, 0.05), photo_thr=(0.05, 0.175, 0.175), lam=0.1,
             z_min=0.1, stop_norm=1e-6, min_rows=10, kahan=False, lm=False) -> IcpOpts:
    it = list(iters) + [0] * (4 - len(iters))
    ep = list(eps) + [0.05] * (4 - len(eps))
    th = list(photo_thr) + [0.175] * (4 - len(photo_thr))
    return IcpOpts(levels, (c_int32 * 4)(*it), (c_float * 4)(*ep), (c_float * 4)(*th), lam, z_min, stop_norm,
                   min_rows, int(kahan), int(lm))


class Icp:
    """ICP context (dtsdf_icp_create / dtsdf_icp_destroy)."""

    def __init__(self, max_width: int, max_height: int, levels: int = 3):
        h = c_void_p()
        check(lib().dtsdf_icp_create(max_width, max_height, levels, ctypes.byref(h)), "dtsdf_icp_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dtsdf_icp_destroy(self._h)
            self._h = None

    __del__ = close

    def set_frame(self, depth, rgb, K, z_min=0.1, z_max=6.0, delta_sup=0.01, stream=None):
        f = Frame(depth.data_ptr(), None if rgb is None else rgb.data_ptr(), intrinsics(K))
        check(lib().dtsdf_icp_set_frame(self._h, ctypes.byref(f), z_min, z_max, delta_sup, _stream_ptr(stream)),
              "dtsdf_icp_set_frame")

    def set_filters(self, f: FilterOpts | None):
        """Bilateral input filters of set_frame (None: off)."""
        check(lib().dtsdf_icp_set_filters(self._h, None if f is None else ctypes.byref(f)), "dtsdf_icp_set_filters")

    def set_keyframe(self, rgb, K, stream=None):
        f = Frame(None, rgb.data_ptr(), intrinsics(K))
        check(lib().dtsdf_icp_set_keyframe(self._h, ctypes.byref(f), _stream_ptr(stream)), "dtsdf_icp_set_keyframe")

    def step(self, ref_depth, ref_normals, K_ref, level, T_rel, opts: IcpOpts, sim3=False, T_rs=None, stream=None,
             raise_on_degenerate=False):
        """One Gauss-Newton iteration; returns (new T_rel, IcpStats)."""
        out = RenderOut(ref_depth.data_ptr(), ref_normals.data_ptr(), None)
        Ki = intrinsics(K_ref)
        T = pose_buf(T_rel)
        st = IcpStats()
        rs = None if T_rs is None else pose_buf(T_rs)
        fn = lib().dtsdf_icp_sim3_step if sim3 else lib().dtsdf_icp_step
        s = fn(self._h, ctypes.byref(out), ctypes.byref(Ki), level, T, rs, ctypes.byref(opts), ctypes.byref(st),
               _stream_ptr(stream))
        if s != OK and (s != ERR_DEGENERATE or raise_on_degenerate):
            check(s, "dtsdf_icp_step")
        return np.array(T[:], np.float64).reshape(4, 4), st

    def solve(self, ref_depth, ref_normals, K_ref, T_rel_dev, opts: IcpOpts, sim3=False, T_rs_dev=None,
              stats_dev=None, stream=None):
        """Whole schedule on the device; T_rel_dev: float64 CUDA tensor [4, 4] updated in place;
        T_rs_dev: float64 CUDA tensor [4, 4] (render -> keyframe camera) or None."""
        out = RenderOut(ref_depth.data_ptr(), ref_normals.data_ptr(), None)
        Ki = intrinsics(K_ref)
        rs = None if T_rs_dev is None else T_rs_dev.data_ptr()
        check(lib().dtsdf_icp_solve(self._h, ctypes.byref(out), ctypes.byref(Ki), int(sim3), T_rel_dev.data_ptr(), rs,
                                    ctypes.byref(opts), None if stats_dev is None else stats_dev.data_ptr(),
                                    _stream_ptr(stream)), "dtsdf_icp_solve")


def _problems(items):
    """items: (icp, ref_normals, K_ref, T_dev, sim3[, stats_dev]) -> ctypes array of IcpProblem."""
    arr = (IcpProblem * max(len(items), 1))()
    for i, it in enumerate(items):
        icp, ref_n, K_ref, T_dev, sim3 = it[:5]
        st = it[5] if len(it) > 5 else None
        arr[i] = IcpProblem(icp._h, RenderOut(None, ref_n.data_ptr(), None), intrinsics(K_ref), T_dev.data_ptr(),
                            None if st is None else st.data_ptr(), int(bool(sim3)))
    return arr


def icp_batch(items, opts: IcpOpts, shape=None, stream=None):
    """Whole geometric schedule for several problems in one launch (dtsdf_icp_batch).
    items: list of (icp: Icp with its frame set, ref_normals CUDA tensor [H, W, 4], K_ref,
    T_dev float64 CUDA tensor [4, 4] updated in place, sim3 bool[, stats_dev uint8 CUDA tensor]);
    shape: (cluster, threads) or None."""
    arr = _problems(items)
    sh = None if shape is None else ctypes.byref(BatchShape(*shape))
    check(lib().dtsdf_icp_batch(arr, len(items), ctypes.byref(opts), sh, _stream_ptr(stream)), "dtsdf_icp_batch")


def icp_batch_tune(items, opts: IcpOpts, stream=None):
    """Fastest (cluster, threads) for these problems and its time in ms (dtsdf_icp_batch_tune)."""
    arr = _problems(items)
    best = BatchShape()
    ms = ctypes.c_float()
    check(lib().dtsdf_icp_batch_tune(arr, len(items), ctypes.byref(opts), ctypes.byref(best), ctypes.byref(ms),
                                     _stream_ptr(stream)), "dtsdf_icp_batch_tune")
    return (best.cluster, best.threads), ms.value


STATS_BYTES = ctypes.sizeof(IcpStats)


def stats_from_device(buf) -> IcpStats:
    """IcpStats from a uint8 CUDA tensor of STATS_BYTES bytes written by the device."""
    st = IcpStats()
    ctypes.memmove(ctypes.byref(st), bytes(buf.cpu().numpy().tobytes()), STATS_BYTES)
    return st


def pose_compose(A_dev, B_dev, C_dev, invert_a=False, stream=None):
    """C = A B (or A^-1 B) on the device for float64 CUDA tensors [4, 4]."""
    check(lib().dtsdf_pose_compose(A_dev.data_ptr(), int(invert_a), B_dev.data_ptr(), C_dev.data_ptr(),
                                   _stream_ptr(stream)), "dtsdf_pose_compose")


def preprocess(depth, K, z_min, z_max, delta_sup, f: FilterOpts | None = None, points=None, normals=None,
               stream=None):
    """Fusion's preprocessing of a float32 CUDA depth image [H, W] (dtsdf_preprocess); returns the
    (points, normals) float32 CUDA tensors [H, W, 4] (w = 1 where present)."""
    import torch
    H, W = depth.shape
    points = torch.empty(H, W, 4, dtype=torch.float32, device=depth.device) if points is None else points
    normals = torch.empty(H, W, 4, dtype=torch.float32, device=depth.device) if normals is None else normals
    fr = Frame(depth.data_ptr(), None, intrinsics(K))
    check(lib().dtsdf_preprocess(ctypes.byref(fr), z_min, z_max, delta_sup, None if f is None else ctypes.byref(f),
                                 points.data_ptr(), normals.data_ptr(), _stream_ptr(stream)), "dtsdf_preprocess")
    return points, normals


def depth_mae(rendered, measured, out=None, stream=None):
    """(sum |rendered - measured|, count) over pixels where both are positive, as a float64 CUDA
    tensor [2] (dtsdf_depth_mae); MAE = out[0] / out[1]."""
    import torch
    if rendered.numel() != measured.numel():
        raise ValueError("rendered / measured: equal sizes")
    out = torch.empty(2, dtype=torch.float64, device=rendered.device) if out is None else out
    check(lib().dtsdf_depth_mae(rendered.data_ptr(), measured.data_ptr(), rendered.numel(), out.data_ptr(),
                                _stream_ptr(stream)), "dtsdf_depth_mae")
    return out


def scale_anchor(log_scale_est, sensor, anchor=0, anchor_log_scale=0.0) -> np.ndarray:
    """Anchored log scales of frames in time order (dtsdf_scale_anchor; host arithmetic)."""
    e = np.ascontiguousarray(log_scale_est, np.float64)
    s = np.ascontiguousarray(sensor, np.int32)
    if e.shape != s.shape or e.ndim != 1:
        raise ValueError("log_scale_est and sensor: equal 1-D shapes")
    out = np.empty_like(e)
    check(lib().dtsdf_scale_anchor(e.ctypes.data, s.ctypes.data, e.shape[0], int(anchor), float(anchor_log_scale),
                                   out.ctypes.data), "dtsdf_scale_anchor")
    return out


def depth_scale(depth_in, depth_out, scale: float, stream=None):
    """depth_out = scale * depth_in on the device (float32 CUDA tensors of equal size)."""
    if depth_in.numel() != depth_out.numel() or depth_in.dtype != depth_out.dtype:
        raise ValueError("depth_in / depth_out: equal float32 sizes")
    check(lib().dtsdf_depth_scale(depth_in.data_ptr(), depth_out.data_ptr(), depth_in.numel(), float(scale),
                                  _stream_ptr(stream)), "dtsdf_depth_scale")


def exp(xi) -> np.ndarray:
    """Device exponential map (se(3) for 6 entries, sim(3) for 7)."""
    x = np.ascontiguousarray(xi, np.float64)
    out = np.zeros(16, np.float64)
    check(lib().dtsdf_exp(1 if x.shape[0] == 7 else 0, x.ctypes.data_as(c_void_p), out.ctypes.data_as(c_void_p)),
          "dtsdf_exp")
    return out.reshape(4, 4)


def server_params(hbm_budget=8 << 30, max_inflight=256, max_batch=32, streams=4, max_width=1280, max_height=720,
                  z_min=0.1, z_max=6.0, delta_sup=0.01, opts: IcpOpts | None = None, shape=(8, 256)) -> ServerParams:
    o = opts if opts is not None else icp_opts(levels=3, iters=(10, 5, 4), eps=(0.01, 0.05, 0.1), lam=0.0)
    return ServerParams(int(hbm_budget), max_inflight, max_batch, streams, max_width, max_height, z_min, z_max,
                        delta_sup, o, BatchShape(*shape))


class Server:
    """Request server over device-resident maps (dtsdf_server_*): submit depth frames with
    prior poses, poll results. Input arrays are kept referenced until their results are polled."""

    def __init__(self, maps, p: ServerParams):
        hs = (c_void_p * len(maps))(*[m._h.value for m in maps])
        h = c_void_p()
        check(lib().dtsdf_server_create(hs, len(maps), ctypes.byref(p), ctypes.byref(h)), "dtsdf_server_create")
        self._h = h
        self._keep = {}
        self.params = p

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().dtsdf_server_destroy(self._h)
            self._h = None
            self._keep = {}

    __del__ = close

    def submit(self, map_index: int, depth: np.ndarray, K, T_prior, sim3=False, tag=0) -> int:
        """depth: host float32 array [H, W] (C-contiguous; pinned memory is copied directly)."""
        d = depth if (isinstance(depth, np.ndarray) and depth.dtype == np.float32 and depth.flags.c_contiguous) \
            else np.ascontiguousarray(depth, np.float32)
        ptr = d.ctypes.data if isinstance(d, np.ndarray) else d.data_ptr()
        r = Request(int(map_index), int(bool(sim3)), intrinsics(K), ptr, pose_buf(T_prior), int(tag))
        seq = ctypes.c_uint64()
        check(lib().dtsdf_server_submit(self._h, ctypes.byref(r), ctypes.byref(seq)), "dtsdf_server_submit")
        self._keep[seq.value] = d
        return seq.value

    def poll(self, cap: int = 64, wait_us: int = 0):
        """Completed results (at most cap); waits up to wait_us for one. A wait that runs out with
        no result returns [] (the library reports DTSDF_ERR_TIMEOUT)."""
        out = (Result * max(cap, 1))()
        n = c_int32()
        st = lib().dtsdf_server_poll(self._h, out, cap, ctypes.byref(n), int(wait_us))
        if st != ERR_TIMEOUT:
            check(st, "dtsdf_server_poll")
        res = [out[i] for i in range(n.value)]
        for r in res:
            self._keep.pop(r.seq, None)
        return res

    def stats(self) -> ServerStats:
        st = ServerStats()
        check(lib().dtsdf_server_stats(self._h, ctypes.byref(st)), "dtsdf_server_stats")
        return st

    def clock(self) -> float:
        return lib().dtsdf_server_clock(self._h)
