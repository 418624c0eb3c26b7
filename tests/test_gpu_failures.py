"""Failure detection on the host, with no GPU fault: the library's error paths under injected
allocation failures, and bounded waits that run out.

With the environment variable DTSDF_FAIL_ALLOC set to N, the N-th device or pinned host
allocation of a create call (counted from 0) and every later one fail as if the device were out
of memory. For every N up to the number of allocations the call makes, dtsdf_create,
dtsdf_icp_create and dtsdf_server_create must return DTSDF_ERR_OOM and free what they had
allocated: the library's count of live allocations (dtsdf_live_allocations) is back where it
was. A server poll whose bounded wait runs out with no result reports DTSDF_ERR_TIMEOUT, and so
does a map whose combine pass had a bounded device wait run out (test hook
DTSDF_TEST_COMBINE_STALL: the pass's producer warp issues nothing)."""
import ctypes
import os

import numpy as np
import pytest
import torch

import paper_2301_12796_gb300 as dt
import scenes
from paper_2301_12796_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    dt.lib()
    yield
    os.environ.pop("DTSDF_FAIL_ALLOC", None)
    os.environ.pop("DTSDF_TEST_COMBINE_STALL", None)


def _walk(create, max_n=64):
    """Fail the N-th allocation for N = 0, 1, ... until the call succeeds; returns the number of
    failing N (the allocations the call makes) and the object of the successful call."""
    L = dt.lib()
    for n in range(max_n):
        live = L.dtsdf_live_allocations()
        os.environ["DTSDF_FAIL_ALLOC"] = str(n)
        try:
            obj = create()
        except dt.DtsdfError as e:
            os.environ.pop("DTSDF_FAIL_ALLOC", None)
            assert e.status == dt.ERR_OOM, (n, e)
            assert L.dtsdf_live_allocations() == live, (n, live, L.dtsdf_live_allocations())
            continue
        os.environ.pop("DTSDF_FAIL_ALLOC", None)
        return n, obj
    raise AssertionError("create kept failing")


def test_map_create_fails_cleanly_at_every_allocation():
    for kw in (dict(voxel_size=0.01, truncation=0.04, max_blocks=1 << 12),
               dict(voxel_size=0.01, truncation=0.04, dense_dim=64, max_blocks=1 << 12),
               dict(voxel_size=0.01, truncation=0.04, max_blocks=1 << 12, storage=dt.STORE_FP16)):
        live = dt.lib().dtsdf_live_allocations()
        n, m = _walk(lambda: dt.Map(dt.params(**kw)))
        assert n >= 10
        m.close()
        torch.cuda.synchronize()
        assert dt.lib().dtsdf_live_allocations() == live


def test_icp_create_fails_cleanly_at_every_allocation():
    live = dt.lib().dtsdf_live_allocations()
    n, ic = _walk(lambda: dt.Icp(320, 240, 3))
    assert n >= 10
    ic.close()
    assert dt.lib().dtsdf_live_allocations() == live


def test_server_create_fails_cleanly_and_bounded_poll_times_out():
    m = dt.Map(dt.params(voxel_size=0.01, truncation=0.04, max_blocks=1 << 12))
    live = dt.lib().dtsdf_live_allocations()
    p = dt.server_params(hbm_budget=64 << 20, max_inflight=8, max_batch=4, streams=2, max_width=320, max_height=240)
    n, srv = _walk(lambda: dt.Server([m], p))
    assert n == 2  # the device arena and the pinned host slots
    # nothing submitted: a bounded wait runs out
    out = (dt.Result * 4)()
    k = ctypes.c_int32(-1)
    st = dt.lib().dtsdf_server_poll(srv._h, out, 4, ctypes.byref(k), 2000)
    assert st == dt.ERR_TIMEOUT and k.value == 0
    assert b"no result" in dt.lib().dtsdf_last_error()
    # a poll that does not wait is not a timeout
    assert dt.lib().dtsdf_server_poll(srv._h, out, 4, ctypes.byref(k), 0) == dt.OK and k.value == 0
    assert srv.poll(4, wait_us=1000) == []
    srv.close()
    assert dt.lib().dtsdf_live_allocations() == live
    m.close()


def test_combine_wait_that_runs_out_is_reported():
    """The combine pass's consumer warps wait for each stage on an mbarrier with a bounded wait
    (2^31 clock cycles). With the producer warp issuing nothing, every such wait runs out (about
    a second): the pass stops, the map's error flags carry bit 4, and the next dtsdf_integrate
    that reads the flags back returns DTSDF_ERR_TIMEOUT. The device stays usable."""
    s = scenes.tiny_scene(1)
    dev = torch.device("cuda:0")
    frames = [s.frame(i) for i in range(4)]
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    m = dt.Map(dt.params(voxel_size=0.01, truncation=0.04, max_blocks=1 << 14, color=True))
    m.integrate(cu(frames[0].depth), cu(frames[0].rgb), s.K, frames[0].pose)
    m.combine(s.K, frames[0].pose, force=True)  # the combined field is allocated by the first call
    torch.cuda.synchronize()
    assert m.stats().error_flags == 0
    os.environ["DTSDF_TEST_COMBINE_STALL"] = "1"
    try:
        m.combine(s.K, frames[0].pose, force=True)
        torch.cuda.synchronize()
    finally:
        os.environ.pop("DTSDF_TEST_COMBINE_STALL", None)
    assert m.stats().error_flags & 16
    with pytest.raises(dt.DtsdfError) as e:
        for f in frames[1:]:
            m.integrate(cu(f.depth), cu(f.rgb), s.K, f.pose)
            torch.cuda.synchronize()
    assert e.value.status == dt.ERR_TIMEOUT
    assert b"bounded device wait" in dt.lib().dtsdf_last_error()
    m.close()
    # the device is still usable: a fresh map fuses, combines and renders
    m2 = dt.Map(dt.params(voxel_size=0.01, truncation=0.04, max_blocks=1 << 14, color=True))
    m2.integrate(cu(frames[0].depth), cu(frames[0].rgb), s.K, frames[0].pose)
    d = torch.zeros(s.K.height, s.K.width, device=dev)
    n = torch.zeros(s.K.height, s.K.width, 4, device=dev)
    m2.render_combined(s.K, frames[0].pose, d, n)
    torch.cuda.synchronize()
    assert m2.stats().error_flags == 0 and (d > 0).float().mean().item() > 0.5
    m2.close()
