"""Edge cases through the C ABI: an empty frame, an empty map, renders of ragged image sizes that
do not fill the 32-ray tiles (1x1, 37x23, 161x97) against the oracle, and registration on an
image too small to give the minimum number of rows (reported degenerate, pose untouched).

Tolerances: the render bar of the parity suite (mask >= 99.9 %, depth within 1e-4 m)."""
import numpy as np
import pytest
import torch

import oracle
import scenes
import paper_2301_12796_gb300 as dt
from paper_2301_12796_gb300 import build as B

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    dt.lib()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _render(gm, K, T):
    d = torch.full((K.height, K.width), 5.0, device=DEV)
    n = torch.full((K.height, K.width, 4), 5.0, device=DEV)
    gm.render(K, T, d, n)
    torch.cuda.synchronize()
    return d.cpu().numpy(), n.cpu().numpy()


def test_empty_frame_and_empty_map():
    s = scenes.tiny_scene(1)
    K = s.K
    gm = dt.Map(dt.params(max_blocks=1 << 12, voxel_size=0.01, truncation=0.04))
    d, n = _render(gm, K, s.poses[0])
    assert not d.any() and not n.any()  # every ray a miss, outputs written
    gm.integrate(torch.zeros(K.height, K.width, device=DEV), None, K, s.poses[0])
    st = gm.stats()
    assert st.bricks == 0 and st.error_flags == 0
    d, n = _render(gm, K, s.poses[0])
    assert not d.any()
    # registration against an empty render: no rows, degenerate, pose untouched
    ic = dt.Icp(K.width, K.height, 1)
    ic.set_frame(cu(s.frame(0).depth), None, K, 0.1, 6.0, 0.02)
    T0 = np.eye(4)
    T1, stt = ic.step(torch.zeros(K.height, K.width, device=DEV), torch.zeros(K.height, K.width, 4, device=DEV), K,
                      0, T0, dt.icp_opts(levels=1, iters=(1,)))
    assert stt.status == dt.ERR_DEGENERATE and stt.rows == 0 and np.array_equal(T1, T0)


@pytest.mark.parametrize("wh", [(1, 1), (37, 23), (161, 97)])
def test_ragged_render_sizes_match_oracle(wh):
    s = scenes.tiny_scene(1)
    om = oracle.OracleMap(oracle.Params(voxel_size=0.01, truncation=0.04, dense_dim=64))
    gm = dt.Map(dt.params(max_blocks=1 << 12, voxel_size=0.01, truncation=0.04, dense_dim=64))
    for i in range(10):
        f = s.frame(i)
        om.integrate(f.depth, f.rgb, s.K, f.pose)
        gm.integrate(cu(f.depth), cu(f.rgb), s.K, f.pose)
    W, H = wh
    # same field of view as the 160x120 sensor, centred
    K = scenes.Intrinsics(W, H, 120.0 * W / 160.0, 120.0 * H / 120.0, (W - 1) / 2.0, (H - 1) / 2.0)
    T = s.poses[5]
    d, n = _render(gm, K, T)
    do, no, _, _ = om.render(K, T)
    assert np.mean((d > 0) == (do > 0)) >= (0.999 if W * H >= 1000 else 1.0)
    both = (d > 0) & (do > 0)
    assert np.all(np.abs(d[both] - do[both]) <= 1e-4)
    assert np.all(n[..., 3][both] == d[both])


def test_icp_on_a_tiny_image_is_degenerate():
    s = scenes.planes_scene()
    K = scenes.Intrinsics(8, 8, 6.0, 6.0, 3.5, 3.5)
    f = s.render(s.poses[0], K=K, noise=False)
    ic = dt.Icp(8, 8, 1)
    ic.set_frame(cu(f.depth), None, K, 0.1, 6.0, 0.02)
    ref = s.render(s.poses[0], K=K, noise=False, exact=True)
    n4 = np.zeros((8, 8, 4), np.float32)
    n4[..., :3] = ref.normals
    n4[..., 3] = ref.depth
    T0 = np.eye(4)
    T1, st = ic.step(cu(ref.depth), cu(n4), K, 0, T0, dt.icp_opts(levels=1, iters=(1,), min_rows=100))
    assert st.status == dt.ERR_DEGENERATE and 0 < st.rows < 100 and np.array_equal(T1, T0)
