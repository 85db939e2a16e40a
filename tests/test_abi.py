"""CPU-side checks of the C ABI boundary: the library builds for sm_103a, loads, and
exports every function include/gp_voxels.h declares; the binding refuses to run without
the library (no fallback).  No compute call is made (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names += re.findall(r"GPV_API\s+[\w\s\*]+?\b(gp\w+)\s*\(", txt)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2410_17084_b300 import build
    return build.build()


def test_header_declares_the_four_named_calls():
    names = declared_functions()
    for n in ("gp_voxels_create", "gp_voxels_insert_scan", "gp_voxels_solve",
              "gp_voxels_init_gaussians"):
        assert n in names, n


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2410_17084_b300 import gp_voxels as g
    assert set(declared_functions()) <= set(g.EXPORTED)


def test_config_layout_matches_binding(libpath):
    """The ctypes struct mirrors gp_voxels_config: the library fills the defaults."""
    from paper_2410_17084_b300 import gp_voxels as g
    cfg = g.gp_voxels_config_default()
    assert abs(cfg.voxel_size - 0.2) < 1e-7 and cfg.n_s == 3 and cfg.n_r == 3 and cfg.tau == 10
    assert cfg.scan_slots == 4 and cfg.max_scan_points == 1 << 17
    assert cfg.lambda_ == 1.0 and cfg.sf2 == 1.0 and abs(cfg.sn2 - 4e-4) < 1e-10


def test_static_calls_without_gpu(libpath):
    from paper_2410_17084_b300 import gp_voxels as g
    assert g.strerror(0) == "ok" and g.strerror(-3) == "memory budget exceeded"
    bad = g.gp_voxels_config_default(grid_side=10)  # n_s * n_r != G
    with pytest.raises(g.GpvError):
        g.gp_voxels_query_sizes(bad)
    cfg = g.gp_voxels_config_default()
    base = g.gp_voxels_query_sizes(cfg)
    assert base > 0
    serve = g.gp_voxels_config_default(hash_capacity=1 << 16)
    assert g.gp_voxels_query_sizes(serve) > base + (1 << 16) * 256 * 12
    with pytest.raises(g.GpvError):  # capacity must be a power of two
        g.gp_voxels_query_sizes(g.gp_voxels_config_default(hash_capacity=1000))


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2410_17084_b300 import gp_voxels as g
    monkeypatch.setattr(g, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(g, "_lib", None)
    with pytest.raises(RuntimeError):
        g.lib()


def test_tensor_core_workspace_split_between_contexts(libpath):
    """The tensor-core variance workspace (tc_workspace_mb) is one total, split evenly between
    the batch entry and the serving scan slots (without the voxel state machine), and a
    memory budget bounds the whole handle."""
    from paper_2410_17084_b300 import gp_voxels as g
    from paper_2410_17084_b300 import serve
    mb = 1 << 20
    for slots in (1, 4):
        off = g.gp_voxels_query_sizes(serve.serving_config(mem_budget=0, scan_slots=slots,
                                                           tc_workspace_mb=0))
        on = g.gp_voxels_query_sizes(serve.serving_config(mem_budget=0, scan_slots=slots))
        lists = ((1 << 16) + slots * (1 << 15)) * 28 + (slots + 1) * 4096
        assert 4095 * mb < on - off <= 4096 * mb + lists
    budgeted = serve.serving_config()
    assert g.gp_voxels_query_sizes(budgeted) <= budgeted.mem_budget
    assert g.gp_voxels_query_sizes(budgeted) > budgeted.mem_budget - 16 * mb
    # with the voxel state machine on, the scan slots keep the CUDA-core variance and the
    # batch entry gets the whole workspace (capped by what max_voxels voxels could use)
    fb = dict(mem_budget=0, eta=0.3, noise_floor=4e-6)
    on = g.gp_voxels_query_sizes(serve.serving_config(**fb))
    off = g.gp_voxels_query_sizes(serve.serving_config(tc_workspace_mb=0, **fb))
    assert 4095 * mb < on - off <= 4096 * mb + (1 << 16) * 28 + 4096
