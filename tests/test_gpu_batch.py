"""Batched registration and batched rendering through the C ABI (dtsdf_icp_batch,
dtsdf_icp_batch_tune, dtsdf_render_batch): parity of every problem of a batch with the FP64
oracle's schedule, independence of the launch shape, uneven image sizes in one batch, and
capture of a whole batch in a CUDA graph.

Tolerances: pose <= 1e-4 rad / 1e-4 m / 1e-5 relative scale against the oracle (as for the
single-problem schedule); different launch shapes sum the same FP32 rows in different orders,
so their poses agree to ~1e-7; a batched render computes every ray exactly as a single render
(bitwise equal)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import icp as oicp
import scenes
import paper_2301_12796_gb300 as dt
from paper_2301_12796_gb300 import build as B

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
EPS = (0.02, 0.2, 0.3)
ITERS = (10, 5, 4)


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    dt.lib()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _ref(scene, T_ref, K):
    ref = scene.render(T_ref, K=K, noise=False, exact=True)
    n4 = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    n4[..., :3] = ref.normals
    n4[..., 3] = ref.depth
    n4[ref.depth == 0] = 0
    return ref.depth, n4


def _problems():
    """Planes-scene problems: SE(3) and Sim(3) (depth scaled), at 160x120 and 320x240."""
    s = scenes.planes_scene()
    K1 = s.K
    K2 = scenes.Intrinsics(320, 240, 240.0, 240.0, 159.5, 119.5)
    out = []
    for i, (K, sim3, scale) in enumerate([(K1, False, 1.0), (K1, True, 1.04), (K2, True, 0.96), (K2, False, 1.0),
                                          (K1, True, 1.0)]):
        rng = np.random.default_rng(40 + i)
        T_ref = s.poses[0] @ scenes.perturbation(rng, 1.0, 0.01)
        T_cur = T_ref @ scenes.perturbation(rng, 2.0, 0.02)
        cur = s.render(T_cur, K=K, noise=True, depth_scale=scale)
        rd, rn = _ref(s, T_ref, K)
        out.append(dict(K=K, sim3=sim3, cur=cur.depth, rd=rd, rn=rn))
    return out


def _oracle_pose(p):
    pre = oracle.preprocess(p["cur"], p["K"], 0.1, 6.0, 0.02)
    levels = oicp.pyramid(pre["z"], p["K"], 3)
    st = oicp.Settings(sim3=p["sim3"], eps=EPS, iters=ITERS)
    To, _ = oicp.track(levels, p["rd"], p["rn"], p["K"], np.eye(4), st)
    return To


def _pose_err(Ta, Tb):
    sa, sb = np.cbrt(np.linalg.det(Ta[:3, :3])), np.cbrt(np.linalg.det(Tb[:3, :3]))
    Ra, Rb = Ta[:3, :3] / sa, Tb[:3, :3] / sb
    ang = np.arccos(np.clip((np.trace(Ra.T @ Rb) - 1) / 2, -1, 1))
    return ang, np.linalg.norm(Ta[:3, 3] - Tb[:3, 3]), abs(sa / sb - 1)


def _setup(probs):
    items, keep = [], []
    for p in probs:
        K = p["K"]
        ic = dt.Icp(K.width, K.height, 3)
        ic.set_frame(cu(p["cur"]), None, K, 0.1, 6.0, 0.02)
        T = torch.eye(4, dtype=torch.float64, device=DEV)
        st = torch.zeros(dt.STATS_BYTES, dtype=torch.uint8, device=DEV)
        rn = cu(p["rn"])
        keep.append((ic, rn))
        items.append((ic, rn, K, T, p["sim3"], st))
    return items, keep


@pytest.fixture(scope="module")
def probs():
    return _problems()


@pytest.fixture(scope="module")
def oracle_poses(probs):
    return [_oracle_pose(p) for p in probs]


@pytest.mark.parametrize("shape", [None, (1, 128), (4, 512), (16, 256)])
def test_icp_batch_matches_oracle(probs, oracle_poses, shape):
    items, keep = _setup(probs)
    opts = dt.icp_opts(levels=3, iters=ITERS, eps=EPS)
    dt.icp_batch(items, opts, shape=shape)
    torch.cuda.synchronize()
    for it, To, p in zip(items, oracle_poses, probs):
        Tg = it[3].cpu().numpy()
        ang, dtr, dsc = _pose_err(Tg, To)
        assert ang <= 1e-4 and dtr <= 1e-4 and dsc <= 1e-5, (p["sim3"], p["K"].width, ang, dtr, dsc)
        st = dt.stats_from_device(it[5])
        assert st.dim == (7 if p["sim3"] else 6) and st.iterations >= 3 and st.status == 0


def test_icp_batch_agrees_with_single_problem_solve(probs):
    items, keep = _setup(probs)
    opts = dt.icp_opts(levels=3, iters=ITERS, eps=EPS)
    dt.icp_batch(items, opts)
    for (ic, rn, K, T, sim3, st), p in zip(items, probs):
        T1 = torch.eye(4, dtype=torch.float64, device=DEV)
        ic.solve(cu(p["rd"]), rn, K, T1, opts, sim3=sim3)
        torch.cuda.synchronize()
        ang, dtr, dsc = _pose_err(T.cpu().numpy(), T1.cpu().numpy())
        assert ang <= 1e-6 and dtr <= 1e-6 and dsc <= 1e-7


def test_icp_batch_tune_keeps_poses(probs):
    items, keep = _setup(probs)
    opts = dt.icp_opts(levels=3, iters=ITERS, eps=EPS)
    (cl, th), ms = dt.icp_batch_tune(items, opts)
    assert cl in (1, 2, 4, 8, 16) and th in (128, 256, 512) and ms > 0
    for it in items:
        assert torch.equal(it[3], torch.eye(4, dtype=torch.float64, device=DEV))


def _tiny_map():
    s = scenes.tiny_scene(1)
    gm = dt.Map(dt.params(max_blocks=1 << 16, voxel_size=0.01, truncation=0.04, dense_dim=64, color=True))
    for i in range(10):
        f = s.frame(i)
        gm.integrate(cu(f.depth), cu(f.rgb), s.K, f.pose)
    return s, gm


def test_render_batch_equals_single_renders():
    s, gm = _tiny_map()
    Ks = [s.K, s.K.scaled(1), scenes.Intrinsics(200, 150, 150.0, 150.0, 99.5, 74.5)]
    jobs, singles = [], []
    for i, K in enumerate(Ks):
        T = s.poses[3 * i] @ scenes.perturbation(np.random.default_rng(i), 1.0, 0.005)
        Td = cu(T)
        outs = [torch.zeros(K.height, K.width, device=DEV), torch.zeros(K.height, K.width, 4, device=DEV),
                torch.zeros(K.height, K.width, 4, device=DEV)]
        jobs.append((K, Td, *outs))
        d = torch.zeros(K.height, K.width, device=DEV)
        n = torch.zeros(K.height, K.width, 4, device=DEV)
        c = torch.zeros(K.height, K.width, 4, device=DEV)
        gm.render_dev(K, Td, d, n, c)
        singles.append((d, n, c))
    gm.render_batch(jobs)
    torch.cuda.synchronize()
    for (K, Td, d, n, c), (d1, n1, c1) in zip(jobs, singles):
        assert (d > 0).float().mean() > 0.5
        assert torch.equal(d, d1) and torch.equal(n, n1) and torch.equal(c, c1)


def test_batch_captured_in_a_cuda_graph(probs):
    """render batch + registration batch in one graph; replays give the eager results."""
    s, gm = _tiny_map()
    K = s.K
    T0 = [cu(s.poses[i]) for i in (0, 5)]
    outs = [(torch.zeros(K.height, K.width, device=DEV), torch.zeros(K.height, K.width, 4, device=DEV)) for _ in T0]
    items, keep = _setup(probs)
    opts = dt.icp_opts(levels=3, iters=ITERS, eps=EPS)
    init = [torch.eye(4, dtype=torch.float64, device=DEV) for _ in items]

    def work(stream):
        for it, e in zip(items, init):
            it[3].copy_(e)
        gm.render_batch([(K, T, d, n, None) for T, (d, n) in zip(T0, outs)], stream=stream)
        dt.icp_batch(items, opts, stream=stream)

    work(torch.cuda.current_stream())
    torch.cuda.synchronize()
    eager = [it[3].clone() for it in items] + [d.clone() for d, _ in outs]
    for it in items:
        it[3].zero_()
    for d, n in outs:
        d.zero_()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            work(side)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        got = [it[3] for it in items] + [d for d, _ in outs]
        for a, b in zip(got, eager):
            assert torch.equal(a, b)


def test_render_launch_shapes_give_identical_outputs():
    """Tile width and refill group only schedule the rays: every shape gives the same bits,
    and the autotuner keeps one of them as the map's shape."""
    s, gm = _tiny_map()
    K = s.K
    T = s.poses[4] @ scenes.perturbation(np.random.default_rng(7), 1.0, 0.005)
    def render():
        d = torch.zeros(K.height, K.width, device=DEV)
        n = torch.zeros(K.height, K.width, 4, device=DEV)
        c = torch.zeros(K.height, K.width, 4, device=DEV)
        gm.render(K, T, d, n, c)
        torch.cuda.synchronize()
        return d, n, c
    ref = render()
    assert (ref[0] > 0).float().mean() > 0.5
    for ctas, refill, tile_w in [(0, 32, 8), (0, 32, 2), (0, 16, 16), (0, 8, 32), (0, 1, 1), (7, 32, 4)]:
        gm.set_render_opts(ctas, refill, tile_w)
        got = render()
        for a, b in zip(got, ref):
            assert torch.equal(a, b), (ctas, refill, tile_w)
    d, n, c = render()
    (ctas, refill, tile_w), ms = gm.tune_render(K, T, d, n, c)
    assert refill in (8, 16, 32) and tile_w in (2, 4, 8, 16, 32) and ms > 0
    for a, b in zip(render(), ref):
        assert torch.equal(a, b)
    with pytest.raises(dt.DtsdfError):
        gm.set_render_opts(0, 3, 8)
    with pytest.raises(dt.DtsdfError):
        gm.set_render_opts(0, 32, 12)
