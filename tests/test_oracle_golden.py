"""The oracle reproduces the golden fixtures of tests/golden (written by make_golden.py from the
oracle alone), and the stored render agrees with the stored analytic plane intersection."""
import os
import sys

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)

import make_golden  # noqa: E402
import oracle  # noqa: E402
from oracle import icp as oicp  # noqa: E402


def load(name):
    return np.loadtxt(os.path.join(HERE, name), comments="#")


def test_plane_render_fixture():
    g = load("plane_render.txt")
    s, m, T = make_golden.plane_case()
    pix = g[:, :2].astype(np.int32)
    d, n, _, _ = m.render(s.K, T, pix)
    assert np.allclose(d, g[:, 2], rtol=0, atol=1e-12)
    assert np.allclose(n, g[:, 3:6], rtol=0, atol=1e-12)
    # the stored values are the analytic ray-plane intersection (Sec. 4 render of a linear field)
    assert np.abs(g[:, 2] - g[:, 6]).max() < 2e-6


def test_plane_icp_fixture():
    g = load("plane_icp.txt")
    s, K, T_ref, T_cur, cur, rd, rn = make_golden.planes_icp_case()
    pre = oracle.preprocess(cur.depth, K, 0.1, 6.0, 0.02)
    levels = oicp.pyramid(pre["z"], K, 3)
    To, _ = oicp.track(levels, rd, rn, K, np.eye(4), oicp.Settings(eps=(0.02, 0.2, 0.3), iters=(10, 5, 4)))
    assert np.allclose(To.ravel(), g[0], rtol=0, atol=1e-12)
    assert np.allclose(g[1], (np.linalg.inv(T_ref) @ T_cur).ravel(), atol=1e-12)
    assert np.abs(g[0] - g[1]).max() < 1e-4
