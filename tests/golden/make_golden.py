"""Writes the golden fixtures of this directory from the FP64 oracle alone (oracle/ and the seeded
scene generator; nothing from the CUDA path).

plane_render.txt  Sec. 4 ray-cast of a fused tilted plane (scenes.plane_scene, 4 frames fused,
                  1 cm voxels, tau 4 cm) at a fixed pose: per pixel u, v, depth, camera-frame
                  normal; the analytic ray-plane intersection is stored beside it.
plane_icp.txt     Secs. 5 / 8 SE(3) schedule (levels 3, iterations 10/5/4) on the planar scene
                  (scenes.planes_scene) from a frame moved by 2 deg / 2 cm: the recovered motion
                  (4x4, row-major) and the true one.

Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import icp as oicp  # noqa: E402
import scenes  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
PIXELS = [(8, 6), (32, 24), (50, 36), (16, 40), (56, 10), (24, 18), (40, 30), (12, 30)]


def plane_case():
    s = scenes.plane_scene()
    m = oracle.OracleMap(oracle.Params(voxel_size=0.01, truncation=0.04))
    for i in range(4):
        f = s.frame(i)
        m.integrate(f.depth, f.rgb, s.K, f.pose)
    T = s.poses[1].copy()
    T[:3, 3] += np.array([0.01, -0.02, 0.01])
    return s, m, T


def planes_icp_case():
    s = scenes.planes_scene()
    K = s.K
    T_ref = s.poses[0]
    rng = np.random.default_rng(5)
    T_cur = T_ref @ scenes.perturbation(rng, 2.0, 0.02)
    cur = s.render(T_cur, noise=False)
    ref = s.render(T_ref, K=K, noise=False, exact=True)
    n4 = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    n4[..., :3] = ref.normals
    n4[..., 3] = ref.depth
    n4[ref.depth == 0] = 0
    return s, K, T_ref, T_cur, cur, ref.depth, n4


def main():
    s, m, T = plane_case()
    pix = np.array(PIXELS, np.int32)
    d, n, _, _ = m.render(s.K, T, pix)
    ex = s.render(T, noise=False, exact=True)
    with open(os.path.join(HERE, "plane_render.txt"), "w") as fh:
        fh.write("# oracle ray-cast (Sec. 4) of the fused tilted plane of scenes.plane_scene(), 4 frames fused,\n")
        fh.write("# 1 cm voxels, tau 4 cm; pose: poses[1] moved by (0.01, -0.02, 0.01) m. Written by make_golden.py.\n")
        fh.write("# u v depth_m nx ny nz analytic_depth_m\n")
        for (u, v), dd, nn in zip(PIXELS, d, n):
            fh.write(f"{u} {v} {dd:.15e} {nn[0]:.15e} {nn[1]:.15e} {nn[2]:.15e} {ex.depth[v, u]:.15e}\n")
    s, K, T_ref, T_cur, cur, rd, rn = planes_icp_case()
    pre = oracle.preprocess(cur.depth, K, 0.1, 6.0, 0.02)
    levels = oicp.pyramid(pre["z"], K, 3)
    st = oicp.Settings(eps=(0.02, 0.2, 0.3), iters=(10, 5, 4))
    To, _ = oicp.track(levels, rd, rn, K, np.eye(4), st)
    true = np.linalg.inv(T_ref) @ T_cur
    with open(os.path.join(HERE, "plane_icp.txt"), "w") as fh:
        fh.write("# oracle SE(3) schedule (Secs. 5, 8; levels 3, iterations 10/5/4, eps 0.02/0.2/0.3) on\n")
        fh.write("# scenes.planes_scene(), current frame moved by 2 deg / 2 cm (seed 5), noise-free; first line\n")
        fh.write("# the recovered current -> reference motion, second line the true one. Written by make_golden.py.\n")
        fh.write(" ".join(f"{x:.15e}" for x in To.ravel()) + "\n")
        fh.write(" ".join(f"{x:.15e}" for x in true.ravel()) + "\n")


if __name__ == "__main__":
    main()
