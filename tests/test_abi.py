"""The C-ABI library loads and exports every entry point include/bvf.h
declares; host-side validation answers without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bvf():
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import bvf as m
    return m


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bvf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bvf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_abi():
    names = declared_functions()
    assert "bvf_run_acoustic" in names and "bvf_transmission" in names
    assert len(names) >= 18


def test_every_declared_symbol_is_exported(bvf):
    lib = bvf.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(bvf.EXPORTS)


def test_version_and_constants(bvf):
    assert bvf.bvf_version() == 2
    assert bvf.bvf_courant_limit() == pytest.approx(6 / (7 * 3 ** 0.5), rel=1e-15)
    assert bvf.lib().bvf_strerror(-2).decode().startswith("time step")


@pytest.mark.parametrize("grid,phys", [
    ((0, 8, 8, 1e-3, 1e-7, 0, 1e-4), (5e5, 1.0, 2)),      # empty grid
    ((8, 8, 8, 1e-3, 1e-7, 4, 1e-4), (5e5, 1.0, 2)),      # too small for the CPML
    ((16, 16, 16, -1e-3, 1e-7, 0, 1e-4), (5e5, 1.0, 2)),  # negative dx
    ((16, 16, 16, 1e-3, 1e-7, 0, 1e-4), (5e5, 1.0, 9)),   # too many SLS mechanisms
    ((16, 16, 16, 1e-3, 1e-7, 0, 1e-4), (-5e5, 1.0, 2)),  # negative f0
    ((16, 16, 16, 1e-3, 1e-7, 2, 2.0), (5e5, 1.0, 2)),    # pml_R outside (0,1)
    ((16, 16, 16, 1e-3, 1e-7, 0, 1e-4), (5e5, 1.0, 2, 7, 0.0)),     # unknown storage
    ((2048, 2048, 512, 1e-3, 1e-7, 0, 1e-4), (5e5, 1.0, 2)),       # 2^31 voxels (32-bit indexing)
    ((16, 16, 16, 1e-3, 1e-7, 0, 1e-4), (5e5, 1.0, 2, 1, -1e5)),    # negative p_ref
])
def test_create_rejects_bad_arguments_on_host(bvf, grid, phys):
    ctx = ctypes.c_void_p()
    rc = bvf.lib().bvf_create(ctypes.byref(bvf.Grid(*grid)), ctypes.byref(bvf.Physics(*phys)),
                              ctypes.byref(ctx))
    assert rc == bvf.BVF_E_ARG and not ctx.value
    assert bvf.lib().bvf_last_error(None)


def test_null_pointers_rejected(bvf):
    L = bvf.lib()
    assert L.bvf_create(None, None, None) == bvf.BVF_E_ARG
    assert L.bvf_rs_plane(None, 4, 4, 1e-3, 0.0, 5e5, None, None) == bvf.BVF_E_ARG
    assert L.bvf_run_acoustic(None, 1, None, None) == bvf.BVF_E_ARG
    assert L.bvf_set_materials(None, None, None, 0) == bvf.BVF_E_ARG
    L.bvf_destroy(None)
