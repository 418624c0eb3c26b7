"""dtsdf_icp_step_noalloc: the ICP iteration for callers that cannot allocate device memory
(real-time loops that cannot afford cudaMalloc's implicit synchronisation, hosts that own all
device memory).

It must give the same normal equations and pose update as the allocating entry points
dtsdf_icp_step / dtsdf_icp_sim3_step (within the tolerances of the other ICP parity tests), in
SE(3) and Sim(3), on consecutive calls that share its fixed scratch. The filtered depth it takes
comes from the library's own preprocessing (dtsdf_preprocess). This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenes
import paper_2301_12796_gb300 as dt
from paper_2301_12796_gb300 import build as B

pytestmark = pytest.mark.gpu


def _stats_from_device(buf):
    return dt.IcpStats.from_buffer_copy(bytes(buf.cpu().numpy().tobytes()))


@pytest.mark.parametrize("sim3", [False, True])
def test_noalloc_step_matches_allocating_step_on_consecutive_calls(sim3):
    B.build()
    L = dt.lib()
    dev = torch.device("cuda:0")
    s = scenes.planes_scene()
    K = s.K
    T_ref = s.poses[0]
    T_cur = T_ref @ scenes.perturbation(np.random.default_rng(17), 2.0, 0.02)
    cur = s.render(T_cur, noise=True, depth_scale=1.03 if sim3 else 1.0)
    ref = s.render(T_ref, noise=False, exact=True)
    rn = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    rn[..., :3] = ref.normals
    rn[..., 3] = ref.depth
    rn[ref.depth == 0] = 0
    rd_t = torch.from_numpy(ref.depth).to(dev)
    rn_t = torch.from_numpy(rn).to(dev)
    z_min, z_max, dsup, eps = 0.1, 6.0, 0.02, 0.05

    # allocating path: context, frame preprocessing, two level-0 iterations
    ic = dt.Icp(K.width, K.height, 1)
    ic.set_frame(torch.from_numpy(cur.depth).to(dev), None, K, z_min, z_max, dsup)
    opts = dt.icp_opts(levels=1, iters=(2,), eps=(eps,), z_min=z_min, min_rows=10)
    T1, st1 = ic.step(rd_t, rn_t, K, 0, np.eye(4), opts, sim3=sim3)
    T2, st2 = ic.step(rd_t, rn_t, K, 0, T1, opts, sim3=sim3)

    # allocation-free path on the same filtered depth, from the library's preprocessing
    P, _ = dt.preprocess(torch.from_numpy(cur.depth).to(dev), K, z_min, z_max, dsup)
    depth_t = torch.where(P[..., 3] > 0, P[..., 2], torch.zeros_like(P[..., 2])).contiguous()
    pose = torch.eye(4, dtype=torch.float64, device=dev)
    stats = torch.zeros(ctypes.sizeof(dt.IcpStats), dtype=torch.uint8, device=dev)
    Ki = dt.intrinsics(K)
    out = dt.RenderOut(rd_t.data_ptr(), rn_t.data_ptr(), None)
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for _ in range(2):
        rc = L.dtsdf_icp_step_noalloc(depth_t.data_ptr(), ctypes.byref(Ki), ctypes.byref(out), ctypes.byref(Ki),
                                      int(sim3), eps, z_min, 10, 1e-6, pose.data_ptr(), stats.data_ptr(), stream)
        assert rc == dt.OK, L.dtsdf_last_error()
        torch.cuda.synchronize()
        results.append((pose.cpu().numpy().copy(), _stats_from_device(stats)))

    for (Tn, sn), (Ta, sa) in zip(results, [(T1, st1), (T2, st2)]):
        assert sn.status == 0 and sa.status == 0
        assert sn.rows == sa.rows
        Hn, Ha = sn.H_matrix(), sa.H_matrix()
        assert np.linalg.norm(Hn - Ha) <= 1e-5 * np.linalg.norm(Ha)
        assert np.allclose(sn.g_vector(), sa.g_vector(), rtol=1e-4, atol=1e-6 * np.abs(sa.g_vector()).max())
        assert np.allclose(Tn, Ta, atol=1e-6)


def test_noalloc_rejects_images_beyond_its_scratch():
    B.build()
    L = dt.lib()
    big = dt.Intrinsics(2048, 1024, 500.0, 500.0, 1023.5, 511.5)
    out = dt.RenderOut(1, 1, None)
    rc = L.dtsdf_icp_step_noalloc(1, ctypes.byref(big), ctypes.byref(out), ctypes.byref(big), 0, 0.05, 0.1, 10, 1e-6,
                                  1, 1, None)
    assert rc == dt.ERR_INVALID_ARG
    assert b"exceeds the fixed scratch" in L.dtsdf_last_error()
