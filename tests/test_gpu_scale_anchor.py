"""Multi-sensor scale anchoring on the device path (Sec. 6, Eq. scale_anchor): a five-sensor cycle
with depth scales (1.0, 1.05, 0.975, 1.025, 0.95), five consecutive frames per sensor, tracked
in Sim(3) against a map, each frame fused after its depth is brought to the model's metric by the
anchored scale (dtsdf_depth_scale) with the SE(3) part of its pose.

Tolerances: the anchored scale of every frame is within 2e-3 (log) of the inverse of its
sensor's depth scale, and the tracked camera within 1 cm / 0.2 deg of the truth; depth scaling is
one rounded float32 product per pixel (bit-exact against numpy's float32 product)."""
import numpy as np
import pytest
import torch

import scenes
import paper_2301_12796_gb300 as dt
from paper_2301_12796_gb300 import build as B

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
CYCLE = (1.0, 1.05, 0.975, 1.025, 0.95)


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    dt.lib()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_depth_scale_is_one_float_product():
    rng = np.random.default_rng(1)
    d = rng.uniform(0.2, 5.0, size=(123, 77)).astype(np.float32)
    d[rng.random(d.shape) < 0.1] = 0
    x = cu(d)
    y = torch.empty_like(x)
    dt.depth_scale(x, y, 1.0 / 1.05)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), d * np.float32(1.0 / 1.05))
    dt.depth_scale(x, x, 2.0)  # in place
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), d * np.float32(2.0))
    with pytest.raises(dt.DtsdfError):
        dt.depth_scale(x, y, -1.0)


def _rot_deg(R):
    return np.degrees(np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)))


def test_five_sensor_cycle_anchored_tracking_and_fusion():
    s = scenes.planes_scene()
    K = s.K
    rng = np.random.default_rng(12)
    # a slow camera path: 0.3 deg / 3 mm per frame
    T = [s.poses[0]]
    for _ in range(34):
        T.append(T[-1] @ scenes.perturbation(rng, 0.3, 0.003))
    sensor = np.repeat(np.tile(np.arange(5), 2), 5)[:35]
    gm = dt.Map(dt.params(max_blocks=1 << 16, voxel_size=0.01, truncation=0.04, color=False))
    for i in range(3):  # the anchor sensor builds the first map at its true poses
        P = T[0] @ scenes.perturbation(rng, 1.0, 0.01)
        gm.integrate(cu(s.render(P, frame_id=100 + i, noise=True).depth), None, K, P)
    ic = dt.Icp(K.width, K.height, 3)
    opts = dt.icp_opts(levels=3, iters=(10, 5, 4), eps=(0.02, 0.1, 0.2), lam=0.0)
    H, W = K.height, K.width
    rd = torch.zeros(H, W, device=DEV)
    rn = torch.zeros(H, W, 4, device=DEV)
    scaled = torch.zeros(H, W, device=DEV)
    est = [T[0]]
    log_est, anchored = [], []
    for k in range(1, 35):
        c = CYCLE[sensor[k]]
        depth = cu(s.render(T[k], frame_id=k, noise=True, depth_scale=c).depth)
        gm.render(K, est[-1], rd, rn)
        ic.set_frame(depth, None, K, 0.1, 6.0, 0.02)
        dT = torch.eye(4, dtype=torch.float64, device=DEV)
        ic.solve(rd, rn, K, dT, opts, sim3=True)
        Tr = dT.cpu().numpy()
        sc = np.cbrt(np.linalg.det(Tr[:3, :3]))
        se3 = Tr.copy()
        se3[:3, :3] /= sc
        est.append(est[-1] @ se3)
        log_est.append(np.log(sc))
        a = dt.scale_anchor(np.array(log_est), sensor[1:k + 1], 0, 0.0)[-1]
        anchored.append(a)
        dt.depth_scale(depth, scaled, float(np.exp(a)))
        gm.integrate(scaled, None, K, est[-1])
        torch.cuda.synchronize()
    anchored = np.array(anchored)
    expect = -np.log(np.array(CYCLE))[sensor[1:]]
    assert np.max(np.abs(anchored - expect)) < 2e-3, np.abs(anchored - expect)
    for k in range(35):
        E = np.linalg.inv(T[k]) @ est[k]
        assert np.linalg.norm(E[:3, 3]) < 0.01 and _rot_deg(E[:3, :3]) < 0.2, k
