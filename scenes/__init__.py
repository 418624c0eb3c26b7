"""Seeded synthetic RGB-D workloads (input generation only).

The paper evaluates on indoor RGB-D sequences (ICL-NUIM, TUM, Zhou; Section 7)
that are not available here. These analytic scenes stand in for them with the
same shapes: 640x480 Kinect-style frames (fx = fy = 525, depth noise
0.0012 z^2 m), rooms with boxes, cylinders and millimetre-thin sheets, seeded
Perlin colour texture, and smooth hand-held-like trajectories.

Nothing in this module computes any part of the DTSDF method: it ray-traces the
ground-truth geometry into depth/RGB images and produces poses. Both the FP64
oracle and the CUDA path consume exactly the arrays produced here.

Workloads:
  * ``tiny``  : 0.64 m box room on a dense 64^3 grid (1 cm voxels, 4 cm
    truncation), a 5 mm plate and a 10 cm (diameter) sphere, ten 160x120 frames
    (fx = fy = 120) on a seeded arc that sees the plate from both sides,
    sigma = 1 mm.
  * ``kinect``: 4 x 4 x 3 m room of seeded boxes, cylinders and 3 mm sheets with
    Perlin RGB, 300 frames at 640x480 (fx = fy = 525, sigma = 0.0012 z^2), a 60
    degree orbit around the central cluster, sensor range 0.1 - 3.0 m.
  * ``sensor_b``: a 1280x720 (fx = fy = 910) view of the kinect room whose depth
    is scaled by a seeded factor in [0.9, 1.1] (multi-sensor Sim(3) case).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libscenegen.so")
_lock = threading.Lock()
_lib = None

PRIM_ROOM, PRIM_BOX, PRIM_CYL, PRIM_SPHERE = 0, 1, 2, 3
PRIM_STRIDE = 24


def build(force: bool = False) -> str:
    """Compile the C ray tracer (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "scenegen.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            D = ctypes.c_double
            P = ctypes.c_void_p
            lib.scene_render.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, D, D, D, D, D,
                                         D, D, D, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                         P, P, P, P, P]
            lib.scene_render.restype = ctypes.c_int
            lib.scene_ray_t.argtypes = [P, ctypes.c_int, P, P]
            lib.scene_ray_t.restype = D
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Intrinsics:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float

    def scaled(self, level: int) -> "Intrinsics":
        """Intrinsics of pyramid level ``level`` (2x2 averaging per level)."""
        k = self
        for _ in range(level):
            k = Intrinsics(k.width // 2, k.height // 2, k.fx / 2.0, k.fy / 2.0,
                           (k.cx - 0.5) / 2.0, (k.cy - 0.5) / 2.0)
        return k


@dataclass
class Frame:
    depth: np.ndarray           # float32 [H, W]
    rgb: np.ndarray             # uint8 [H, W, 3]
    pose: np.ndarray            # float64 [4, 4] camera-to-world
    K: Intrinsics
    points: np.ndarray | None = None   # float64 [H, W, 3] exact camera-frame points
    normals: np.ndarray | None = None  # float64 [H, W, 3] exact camera-frame normals
    ids: np.ndarray | None = None


@dataclass
class Scene:
    name: str
    prims: np.ndarray                 # float64 [n, 24]
    K: Intrinsics
    poses: list                       # camera-to-world 4x4 per frame
    noise_s0: float
    noise_s2: float
    z_min: float
    z_max: float
    seed: int
    tex_seed: int
    extra: dict = field(default_factory=dict)

    @property
    def n_frames(self) -> int:
        return len(self.poses)

    def render(self, pose: np.ndarray, K: Intrinsics | None = None, frame_id: int = 0,
               noise: bool = True, exact: bool = False, depth_scale: float = 1.0) -> Frame:
        """Ray-trace the scene at ``pose``; ``depth_scale`` multiplies the depth
        (a sensor with a wrong metric scale, as in the multi-sensor case)."""
        lib = _load()
        K = K or self.K
        H, W = K.height, K.width
        depth = np.zeros((H, W), np.float32)
        rgb = np.zeros((H, W, 3), np.uint8)
        pts = np.zeros((H, W, 3), np.float64) if exact else None
        nrm = np.zeros((H, W, 3), np.float64) if exact else None
        ids = np.zeros((H, W), np.int32) if exact else None
        T = np.ascontiguousarray(pose, np.float64)
        prims = np.ascontiguousarray(self.prims, np.float64)
        s0, s2 = (self.noise_s0, self.noise_s2) if noise else (0.0, 0.0)
        zmin, zmax = self.z_min / depth_scale, self.z_max / depth_scale
        lib.scene_render(_ptr(prims), prims.shape[0], _ptr(T), W, H, K.fx, K.fy, K.cx, K.cy,
                         s0, s2, zmin, zmax, self.seed, frame_id, self.tex_seed,
                         _ptr(depth), _ptr(rgb), _ptr(pts), _ptr(nrm), _ptr(ids))
        if depth_scale != 1.0:
            depth = (depth.astype(np.float64) * depth_scale).astype(np.float32)
            if pts is not None:
                pts = pts * depth_scale
        return Frame(depth, rgb, T.copy(), K, pts, nrm, ids)

    def frame(self, i: int, exact: bool = False) -> Frame:
        return self.render(self.poses[i], frame_id=i, exact=exact)

    def ray_t(self, origin, direction) -> float:
        lib = _load()
        o = np.ascontiguousarray(origin, np.float64)
        d = np.ascontiguousarray(direction, np.float64)
        prims = np.ascontiguousarray(self.prims, np.float64)
        return lib.scene_ray_t(_ptr(prims), prims.shape[0], _ptr(o), _ptr(d))


# ------------------------------------------------------------------ poses --

def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world pose with the camera z axis toward ``target`` and y down."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    if np.linalg.norm(x) < 1e-9:
        x = np.cross(z, np.array([0.0, 1.0, 0.0]))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = x, y, z, eye
    return T


def _rodrigues(w) -> np.ndarray:
    w = np.asarray(w, np.float64)
    th = np.linalg.norm(w)
    if th < 1e-15:
        return np.eye(3)
    k = w / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx


def perturbation(rng: np.random.Generator, angle_deg: float, trans_m: float) -> np.ndarray:
    """Rigid transform with a seeded axis, the given rotation angle and translation length."""
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    t = rng.normal(size=3)
    t /= np.linalg.norm(t)
    T = np.eye(4)
    T[:3, :3] = _rodrigues(a * np.deg2rad(angle_deg))
    T[:3, 3] = t * trans_m
    return T


# ---------------------------------------------------------------- scenes --

def _prim(kind, oid, a, b, R=None, colA=(0, 0, 0), colB=(255, 255, 255), freq=4.0):
    p = np.zeros(PRIM_STRIDE)
    p[0], p[1] = kind, oid
    p[2:5] = np.pad(np.asarray(a, np.float64), (0, 3 - len(a)))
    p[5:8] = np.pad(np.asarray(b, np.float64), (0, 3 - len(b)))
    p[8:17] = (np.eye(3) if R is None else np.asarray(R)).reshape(-1)
    p[17:20], p[20:23], p[23] = colA, colB, freq
    return p


def _yaw(phi):
    c, s = np.cos(phi), np.sin(phi)
    # rows are the box axes expressed in world coordinates
    return np.array([[c, s, 0.0], [-s, c, 0.0], [0.0, 0.0, 1.0]])


def tiny_scene(seed: int = 1, n_frames: int = 10) -> Scene:
    """0.64 m box room (interior faces at 0.04 / 0.59 m), 5 mm plate, r = 5 cm sphere."""
    rng = np.random.default_rng(seed)
    prims = [
        _prim(PRIM_ROOM, 0, (0.04, 0.04, 0.04), (0.59, 0.59, 0.59), colA=(90, 80, 70), colB=(200, 190, 170), freq=12),
        # the plate: 5 mm thick along x, seen from both sides by the arc
        _prim(PRIM_BOX, 1, (0.3140, 0.315, 0.27), (0.0025, 0.12, 0.13), colA=(20, 60, 160), colB=(220, 220, 60), freq=20),
        _prim(PRIM_SPHERE, 2, (0.43, 0.46, 0.16), (0.05,), colA=(160, 30, 30), colB=(250, 160, 120), freq=25),
    ]
    K = Intrinsics(160, 120, 120.0, 120.0, 80.0, 60.0)
    centre = np.array([0.315, 0.315, 0.27])
    poses = []
    for k in range(n_frames):
        phi = np.deg2rad(-150.0 + 300.0 * k / max(n_frames - 1, 1) + rng.uniform(-4, 4))
        r = 0.21 + rng.uniform(-0.01, 0.01)
        eye = centre + np.array([-r * np.cos(phi), -r * np.sin(phi), 0.06 + rng.uniform(-0.01, 0.01)])
        target = centre + rng.uniform(-0.01, 0.01, size=3)
        poses.append(look_at(eye, target))
    return Scene("tiny", np.stack(prims), K, poses, noise_s0=0.001, noise_s2=0.0, z_min=0.1, z_max=6.0,
                 seed=seed, tex_seed=seed + 1000)


def _palette(rng):
    a = rng.integers(10, 140, size=3)
    b = rng.integers(120, 250, size=3)
    return tuple(float(x) for x in a), tuple(float(x) for x in b), float(rng.uniform(3.0, 9.0))


def kinect_room(seed: int = 1, n_frames: int = 300, arc_deg: float = 60.0, z_max: float = 3.0) -> Scene:
    """4 x 4 x 3 m room of seeded boxes, cylinders and 3 mm sheets, 640x480 Kinect frames."""
    rng = np.random.default_rng(seed)
    prims = []
    cA, cB, f = _palette(rng)
    prims.append(_prim(PRIM_ROOM, 0, (0.0, 0.0, 0.0), (4.0, 4.0, 3.0), colA=cA, colB=cB, freq=f))
    oid = 1
    C = np.array([2.0, 2.0])
    # central cluster, seen from all sides along the orbit: thin sheets, a cylinder, a box
    for k in range(3):
        ang = rng.uniform(0, 2 * np.pi)
        pos = C + rng.uniform(0.05, 0.35) * np.array([np.cos(ang), np.sin(ang)])
        w, h = rng.uniform(0.35, 0.6), rng.uniform(0.5, 0.9)
        z0 = rng.uniform(0.5, 0.9)
        cA, cB, f = _palette(rng)
        prims.append(_prim(PRIM_BOX, oid, (pos[0], pos[1], z0 + h), (0.0015, w, h), R=_yaw(rng.uniform(0, np.pi)),
                           colA=cA, colB=cB, freq=f))
        oid += 1
    cA, cB, f = _palette(rng)
    prims.append(_prim(PRIM_CYL, oid, (C[0] + 0.25, C[1] - 0.3, 0.0), (0.12, 0.0, 1.1), colA=cA, colB=cB, freq=f))
    oid += 1
    cA, cB, f = _palette(rng)
    prims.append(_prim(PRIM_BOX, oid, (C[0] - 0.25, C[1] + 0.2, 0.25), (0.22, 0.18, 0.25), R=_yaw(rng.uniform(0, np.pi)),
                       colA=cA, colB=cB, freq=f))
    oid += 1
    # furniture along the walls
    for k in range(8):
        side = k % 4
        s = rng.uniform(0.5, 3.5)
        depth_in = rng.uniform(0.3, 0.6)
        pos = [(s, depth_in), (4 - depth_in, s), (s, 4 - depth_in), (depth_in, s)][side]
        e = (rng.uniform(0.15, 0.45), rng.uniform(0.15, 0.35), rng.uniform(0.2, 0.6))
        cA, cB, f = _palette(rng)
        prims.append(_prim(PRIM_BOX, oid, (pos[0], pos[1], e[2]), e, R=_yaw(rng.uniform(0, np.pi)), colA=cA, colB=cB, freq=f))
        oid += 1
    for k in range(4):
        side = (k + 1) % 4
        s = rng.uniform(0.5, 3.5)
        pos = [(s, 0.35), (3.65, s), (s, 3.65), (0.35, s)][side]
        cA, cB, f = _palette(rng)
        prims.append(_prim(PRIM_CYL, oid, (pos[0], pos[1], 0.0), (rng.uniform(0.08, 0.2), 0.0, rng.uniform(0.6, 2.0)),
                           colA=cA, colB=cB, freq=f))
        oid += 1
    for k in range(3):
        side = (k + 2) % 4
        s = rng.uniform(0.8, 3.2)
        pos = [(s, 0.9), (3.1, s), (s, 3.1), (0.9, s)][side]
        cA, cB, f = _palette(rng)
        w, h = rng.uniform(0.3, 0.6), rng.uniform(0.4, 0.8)
        prims.append(_prim(PRIM_BOX, oid, (pos[0], pos[1], 0.3 + h), (0.0015, w, h), R=_yaw(rng.uniform(0, np.pi)),
                           colA=cA, colB=cB, freq=f))
        oid += 1
    cA, cB, f = _palette(rng)
    prims.append(_prim(PRIM_SPHERE, oid, (C[0] + 0.5, C[1] + 0.45, 0.2), (0.2,), colA=cA, colB=cB, freq=f))

    K = Intrinsics(640, 480, 525.0, 525.0, 319.5, 239.5)
    # orbit around the central cluster, looking inward with a slow seeded wobble
    poses = []
    ph0 = rng.uniform(0, 2 * np.pi)
    wob = rng.uniform(0, 2 * np.pi, size=4)
    for i in range(n_frames):
        s = i / max(n_frames - 1, 1)
        ph = ph0 + np.deg2rad(arc_deg) * s
        r = 1.35 + 0.1 * np.sin(2 * np.pi * s + wob[0])
        eye = np.array([C[0] + r * np.cos(ph), C[1] + r * np.sin(ph), 1.45 + 0.08 * np.sin(3 * np.pi * s + wob[1])])
        target = np.array([C[0] + 0.25 * np.sin(2 * np.pi * s + wob[2]), C[1] + 0.25 * np.cos(2 * np.pi * s + wob[3]),
                           0.9 + 0.1 * np.sin(4 * np.pi * s)])
        poses.append(look_at(eye, target))
    return Scene("kinect", np.stack(prims), K, poses, noise_s0=0.0, noise_s2=0.0012, z_min=0.1, z_max=z_max,
                 seed=seed, tex_seed=seed + 1000)


def sensor_b(room: Scene, seed: int = 1) -> tuple[Intrinsics, float, np.random.Generator]:
    """Second sensor of the multi-sensor case: 1280x720, fx = fy = 910, seeded depth scale."""
    rng = np.random.default_rng(seed + 7777)
    scale = float(rng.uniform(0.9, 1.1))
    return Intrinsics(1280, 720, 910.0, 910.0, 639.5, 359.5), scale, rng


def multi_sensor_problems(room: Scene, n: int = 64, seed: int = 1, rot_deg: float = 5.0,
                          trans_m: float = 0.10) -> list[dict]:
    """n registrations of the second sensor (sensor_b) against a map of ``room`` built from the
    first sensor: true pose near the first sensor's trajectory, seeded depth scale, prior = the
    true pose perturbed by rot_deg degrees and trans_m metres."""
    out = []
    for i in range(n):
        K, scale, rng = sensor_b(room, seed + i)
        T_true = room.poses[(i * len(room.poses)) // n] @ perturbation(rng, 2.0, 0.05)
        frame = room.render(T_true, K=K, frame_id=100000 + i, noise=True, depth_scale=scale)
        prior = T_true @ perturbation(rng, rot_deg, trans_m)
        out.append(dict(K=K, scale=scale, T_true=T_true, prior=prior, depth=frame.depth))
    return out


def planes_scene(seed: int = 3) -> Scene:
    """Only planar surfaces (room corner and a tilted box): point-to-plane ICP
    has its exact optimum at the true pose on such a scene."""
    rng = np.random.default_rng(seed)
    prims = [
        _prim(PRIM_ROOM, 0, (0.0, 0.0, 0.0), (2.0, 2.0, 2.0), colA=(40, 90, 140), colB=(230, 200, 120), freq=5),
        _prim(PRIM_BOX, 1, (0.6, 0.7, 0.3), (0.25, 0.2, 0.3), R=_yaw(0.6), colA=(150, 40, 40), colB=(250, 220, 90),
              freq=9),
        _prim(PRIM_BOX, 2, (1.2, 0.4, 0.5), (0.15, 0.3, 0.5), R=_yaw(-0.3), colA=(30, 140, 60), colB=(210, 240, 230),
              freq=7),
    ]
    K = Intrinsics(160, 120, 120.0, 120.0, 79.5, 59.5)
    eye = np.array([1.7, 1.6, 1.3]) + rng.uniform(-0.05, 0.05, size=3)
    poses = [look_at(eye, np.array([0.5, 0.5, 0.4]))]
    return Scene("planes", np.stack(prims), K, poses, noise_s0=0.0, noise_s2=0.0, z_min=0.1, z_max=6.0,
                 seed=seed, tex_seed=seed + 1000)


def plane_scene(normal=(0.3, -0.2, 1.0), offset: float = 0.0, seed: int = 5) -> Scene:
    """A single large tilted slab whose top face is the plane <n, x> = offset."""
    n = np.asarray(normal, np.float64)
    n /= np.linalg.norm(n)
    # box axes: rows of R; third axis along n
    a = np.cross(n, [1.0, 0.0, 0.0])
    if np.linalg.norm(a) < 1e-6:
        a = np.cross(n, [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(n, a)
    R = np.stack([a, b, n])
    centre = n * (offset - 0.5)
    prims = [_prim(PRIM_BOX, 0, centre, (3.0, 3.0, 0.5), R=R, colA=(60, 60, 60), colB=(200, 120, 40), freq=6)]
    K = Intrinsics(64, 48, 50.0, 50.0, 31.5, 23.5)
    rng = np.random.default_rng(seed)
    poses = []
    for k in range(4):
        eye = n * (0.8 + 0.1 * k) + a * rng.uniform(-0.2, 0.2) + b * rng.uniform(-0.2, 0.2)
        poses.append(look_at(eye, n * offset + a * rng.uniform(-0.05, 0.05), up=tuple(b)))
    return Scene("plane", np.stack(prims), K, poses, noise_s0=0.0, noise_s2=0.0, z_min=0.1, z_max=6.0,
                 seed=seed, tex_seed=seed + 1000, extra=dict(normal=n, offset=offset))


# ---------------------------------------------------------------- serving --

# sensor classes of the serving workload and their shares of the requests
SERVE_SENSORS = (
    (Intrinsics(320, 240, 262.5, 262.5, 159.5, 119.5), 0.3),
    (Intrinsics(640, 480, 525.0, 525.0, 319.5, 239.5), 0.5),
    (Intrinsics(1280, 720, 910.0, 910.0, 639.5, 359.5), 0.2),
)


def serve_requests(rooms: list, n: int, seed: int = 1, rate: float = 2000.0, sim3_every: int = 4,
                   rot_deg: float = 2.0, trans_m: float = 0.02, pool: int | None = None) -> list[dict]:
    """n render + registration requests against maps of ``rooms``: Poisson arrival times at
    ``rate`` per second (key t, seconds), the map drawn uniformly, the sensor drawn with the
    SERVE_SENSORS shares, every ``sim3_every``-th request a Sim(3) one whose depth is scaled by a
    seeded factor in [0.9, 1.1]; the true pose is a seeded frame of the room's trajectory moved
    by 2 deg / 5 cm, the prior that pose perturbed by rot_deg / trans_m. With ``pool`` the frames
    of the first ``pool`` requests are reused cyclically by the later ones (same map, sensor,
    kind, poses and depth), so long request streams need few ray-traced frames."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
    shares = np.array([w for _, w in SERVE_SENSORS])
    out = []
    for i in range(n):
        if pool is not None and i >= pool:
            q = dict(out[i % pool])
            q["t"] = float(arrivals[i])
            out.append(q)
            continue
        mi = int(rng.integers(len(rooms)))
        room = rooms[mi]
        K = SERVE_SENSORS[int(rng.choice(len(SERVE_SENSORS), p=shares))][0]
        sim3 = (i % sim3_every) == sim3_every - 1
        scale = float(rng.uniform(0.9, 1.1)) if sim3 else 1.0
        T_true = room.poses[int(rng.integers(room.n_frames))] @ perturbation(rng, 2.0, 0.05)
        frame = room.render(T_true, K=K, frame_id=200000 + i, noise=True, depth_scale=scale)
        prior = T_true @ perturbation(rng, rot_deg, trans_m)
        out.append(dict(t=float(arrivals[i]), map=mi, K=K, sim3=sim3, scale=scale, T_true=T_true, prior=prior,
                        depth=frame.depth))
    return out
