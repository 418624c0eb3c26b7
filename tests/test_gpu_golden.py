"""The device path against the golden fixtures of tests/golden (oracle values written by
make_golden.py): the render of the fused tilted plane (depth <= 1e-4 m, normal <= 1e-3 rad) and
the SE(3) schedule on the planar scene (pose <= 1e-4 rad / 1e-4 m)."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)

import angles  # noqa: E402
import make_golden  # noqa: E402
import paper_2301_12796_gb300 as dt  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_device_render_matches_golden_plane():
    g = np.loadtxt(os.path.join(HERE, "plane_render.txt"), comments="#")
    s = make_golden.scenes.plane_scene()
    gm = dt.Map(dt.params(voxel_size=0.01, truncation=0.04, max_blocks=1 << 14))
    for i in range(4):
        f = s.frame(i)
        gm.integrate(cu(f.depth), cu(f.rgb), s.K, f.pose)
    T = s.poses[1].copy()
    T[:3, 3] += np.array([0.01, -0.02, 0.01])
    d = torch.zeros(s.K.height, s.K.width, device=DEV)
    n = torch.zeros(s.K.height, s.K.width, 4, device=DEV)
    gm.render(s.K, T, d, n)
    torch.cuda.synchronize()
    d, n = d.cpu().numpy(), n.cpu().numpy()
    u, v = g[:, 0].astype(int), g[:, 1].astype(int)
    assert np.abs(d[v, u] - g[:, 2]).max() <= 1e-4
    ang = angles.between(n[v, u, :3], g[:, 3:6])
    assert ang.max() <= 1e-3
    gm.close()


def test_device_registration_matches_golden_plane():
    g = np.loadtxt(os.path.join(HERE, "plane_icp.txt"), comments="#")
    s, K, T_ref, T_cur, cur, rd, rn = make_golden.planes_icp_case()
    ic = dt.Icp(K.width, K.height, 3)
    ic.set_frame(cu(cur.depth), None, K, 0.1, 6.0, 0.02)
    Tdev = torch.eye(4, dtype=torch.float64, device=DEV)
    ic.solve(cu(rd), cu(rn), K, Tdev, dt.icp_opts(levels=3, iters=(10, 5, 4), eps=(0.02, 0.2, 0.3), lam=0.0))
    Tg = Tdev.cpu().numpy()
    To = g[0].reshape(4, 4)
    ang = np.arccos(np.clip((np.trace(Tg[:3, :3].T @ To[:3, :3]) - 1) / 2, -1, 1))
    assert ang <= 1e-4 and np.linalg.norm(Tg[:3, 3] - To[:3, 3]) <= 1e-4
    ic.close()
