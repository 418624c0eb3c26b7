"""The C ABI library loads and exports every symbol include/dtsdf.h declares, and the
Python binding's struct layouts match the header (no GPU needed)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

import paper_2301_12796_gb300 as dt
from paper_2301_12796_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dtsdf.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return dt.lib()


def declared_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"DTSDF_API\s+[\w\s\*]+?\b(dtsdf_\w+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dtsdf_create", "dtsdf_integrate", "dtsdf_render", "dtsdf_icp_step", "dtsdf_icp_sim3_step"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (dtsdf_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    assert set(declared_functions()) == set(dt.SIGNATURES)


def test_struct_layouts_match_header():
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "dtsdf.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(dtsdf_params), sizeof(dtsdf_intrinsics),
             sizeof(dtsdf_frame), sizeof(dtsdf_render_out), sizeof(dtsdf_map_stats_t),
             sizeof(dtsdf_icp_opts), sizeof(dtsdf_icp_stats));
      printf("%zu %zu %zu %zu\n", offsetof(dtsdf_icp_opts, stop_norm), offsetof(dtsdf_icp_stats, rows),
             offsetof(dtsdf_params, max_blocks), offsetof(dtsdf_icp_opts, lm));
      printf("%zu %zu %zu %zu\n", sizeof(dtsdf_render_opts), sizeof(dtsdf_icp_problem), sizeof(dtsdf_batch_shape),
             sizeof(dtsdf_render_job));
      printf("%zu %zu %zu\n", offsetof(dtsdf_icp_problem, K_ref), offsetof(dtsdf_icp_problem, sim3),
             offsetof(dtsdf_render_job, out));
      printf("%zu %zu %zu %zu\n", sizeof(dtsdf_server_params), sizeof(dtsdf_request), sizeof(dtsdf_result),
             sizeof(dtsdf_server_stats_t));
      printf("%zu %zu %zu %zu\n", offsetof(dtsdf_server_params, opts), offsetof(dtsdf_server_params, shape),
             offsetof(dtsdf_request, T_prior), offsetof(dtsdf_result, stats));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(x) for x in lines[0].split()]
    offs = [int(x) for x in lines[1].split()]
    assert sizes == [ctypes.sizeof(x) for x in (dt.Params, dt.Intrinsics, dt.Frame, dt.RenderOut, dt.MapStats,
                                                dt.IcpOpts, dt.IcpStats)]
    assert offs == [dt.IcpOpts.stop_norm.offset, dt.IcpStats.rows.offset, dt.Params.max_blocks.offset,
                    dt.IcpOpts.lm.offset]
    assert [int(x) for x in lines[2].split()] == [ctypes.sizeof(x) for x in (dt.RenderOpts, dt.IcpProblem,
                                                                             dt.BatchShape, dt.RenderJob)]
    assert [int(x) for x in lines[3].split()] == [dt.IcpProblem.K_ref.offset, dt.IcpProblem.sim3.offset,
                                                  dt.RenderJob.out.offset]
    assert [int(x) for x in lines[4].split()] == [ctypes.sizeof(x) for x in (dt.ServerParams, dt.Request, dt.Result,
                                                                             dt.ServerStats)]
    assert [int(x) for x in lines[5].split()] == [dt.ServerParams.opts.offset, dt.ServerParams.shape.offset,
                                                  dt.Request.T_prior.offset, dt.Result.stats.offset]


def test_invalid_parameters_rejected_on_host(lib):
    # argument checks run before any CUDA call
    h = ctypes.c_void_p()
    bad = dt.params(voxel_size=-1.0)
    assert lib.dtsdf_create(ctypes.byref(bad), None, ctypes.byref(h)) == dt.ERR_INVALID_ARG
    bad = dt.params(theta=0.5)  # below acos(1/sqrt(3)): some normals would belong to no direction
    assert lib.dtsdf_create(ctypes.byref(bad), None, ctypes.byref(h)) == dt.ERR_INVALID_ARG
    bad = dt.params(dense_dim=60)
    assert lib.dtsdf_create(ctypes.byref(bad), None, ctypes.byref(h)) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_create(None, None, ctypes.byref(h)) == dt.ERR_INVALID_ARG
    assert b"invalid" in lib.dtsdf_last_error() or b"null" in lib.dtsdf_last_error()
    assert lib.dtsdf_icp_create(4, 4, 3, ctypes.byref(h)) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_icp_create(640, 480, 9, ctypes.byref(h)) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_destroy(None) == dt.ERR_INVALID_ARG
    # batch entry points check their arguments before any CUDA call
    opts = dt.icp_opts()
    assert lib.dtsdf_icp_batch(None, 1, ctypes.byref(opts), None, None) == dt.ERR_INVALID_ARG
    pr = (dt.IcpProblem * 1)()
    assert lib.dtsdf_icp_batch(pr, 1, ctypes.byref(opts), None, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_icp_batch(pr, 0, ctypes.byref(opts), ctypes.byref(dt.BatchShape(3, 256)), None) == \
        dt.ERR_INVALID_ARG
    assert lib.dtsdf_render_batch(None, None, 1, None) == dt.ERR_INVALID_ARG
    # Levenberg-Marquardt is an option of the single-problem schedule only
    lm = dt.icp_opts(lm=True)
    assert lib.dtsdf_icp_batch(pr, 0, ctypes.byref(lm), None, None) == dt.ERR_INVALID_ARG
    # the server checks its parameters before allocating anything
    sp = dt.server_params(hbm_budget=0)
    maps = (ctypes.c_void_p * 1)(1)
    assert lib.dtsdf_server_create(maps, 1, ctypes.byref(sp), ctypes.byref(h)) == dt.ERR_INVALID_ARG
    sp = dt.server_params(streams=99)
    assert lib.dtsdf_server_create(maps, 1, ctypes.byref(sp), ctypes.byref(h)) == dt.ERR_INVALID_ARG
    sp = dt.server_params(opts=dt.icp_opts(lm=True))
    assert lib.dtsdf_server_create(maps, 1, ctypes.byref(sp), ctypes.byref(h)) == dt.ERR_INVALID_ARG
    sp = dt.server_params(shape=(3, 256))
    assert lib.dtsdf_server_create(maps, 1, ctypes.byref(sp), ctypes.byref(h)) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_server_create(None, 1, ctypes.byref(dt.server_params()), ctypes.byref(h)) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_server_submit(None, None, None) == dt.ERR_INVALID_ARG
    # the later entry points: argument checks before any CUDA call
    assert lib.dtsdf_recycle(None, 0.75, None, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_render_freespace(None, None, None, None, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_set_filters(None, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_icp_set_filters(None, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_preprocess(None, 0.1, 6.0, 0.02, None, None, None, None) == dt.ERR_INVALID_ARG
    fr = dt.Frame(1, None, dt.intrinsics(__import__("scenes").Intrinsics(8, 8, 6.0, 6.0, 3.5, 3.5)))
    bad = dt.filter_opts(depth_radius=9)
    assert lib.dtsdf_preprocess(ctypes.byref(fr), 0.1, 6.0, 0.02, ctypes.byref(bad), 1, 1, None) == dt.ERR_INVALID_ARG
    bad = dt.filter_opts(normal_sigma_r=0.0)
    assert lib.dtsdf_preprocess(ctypes.byref(fr), 0.1, 6.0, 0.02, ctypes.byref(bad), 1, 1, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_depth_mae(None, None, 4, None, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_depth_scale(None, None, 4, 1.0, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_depth_scale(1, 1, 4, -1.0, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_depth_scale(1, 1, 4, float("inf"), None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_scale_anchor(None, None, 3, 0, 0.0, None) == dt.ERR_INVALID_ARG
    assert lib.dtsdf_scale_anchor(None, None, 0, 0, 0.0, None) == dt.OK


def test_product_path_has_no_cpu_fallback(tmp_path, monkeypatch):
    # with the shared library absent the binding raises instead of computing anything itself
    monkeypatch.setattr(dt, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(dt, "_lib", None)
    with pytest.raises(RuntimeError):
        dt.lib()


def test_package_does_not_import_oracle():
    import sys
    src = open(os.path.join(ROOT, "paper_2301_12796_gb300", "__init__.py")).read()
    assert "oracle" not in re.findall(r"^\s*(?:import|from)\s+(\w+)", src, flags=re.M)
    for f in os.listdir(os.path.join(ROOT, "paper_2301_12796_gb300", "csrc")):
        assert "oracle" not in open(os.path.join(ROOT, "paper_2301_12796_gb300", "csrc", f)).read()
