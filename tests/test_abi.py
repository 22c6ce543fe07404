"""The C-ABI library loads and exports every entry point include/bvf.h and
include/bvf_fno.h declare; host-side validation answers without touching a
GPU."""
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


def declared_functions(header="bvf.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
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


def test_surrogate_header_symbols_are_exported(bvf):
    from paper_2301_12727_gb300 import fno
    names = declared_functions("bvf_fno.h")
    assert "bvf_fno_forward" in names
    lib = fno.lib()
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(fno.EXPORTS)


def test_surrogate_validation_on_host(bvf):
    from oracle import fno as ofno
    from paper_2301_12727_gb300 import fno
    good = dict(c_in=8, width=32, modes=12, n_layers=4, hidden=128, c_out=1)
    assert fno.bvf_fno_weight_count(fno.FnoDims(**good)) == ofno.weight_count(**good)
    for bad in (dict(good, width=30), dict(good, width=128), dict(good, width=8),
                dict(good, width=20), dict(good, modes=0),
                dict(good, modes=17), dict(good, c_in=17), dict(good, hidden=0),
                dict(good, c_out=9), dict(good, n_layers=0)):
        assert fno.bvf_fno_weight_count(fno.FnoDims(**bad)) == 0
    L = fno.lib()
    h = ctypes.c_void_p()
    d = fno.FnoDims(**good)
    w = (ctypes.c_float * 4)()
    assert L.bvf_fno_create(ctypes.byref(h), ctypes.byref(d), w, 4) == bvf.BVF_E_ARG
    assert not h.value and L.bvf_last_error(None)
    assert L.bvf_fno_create(ctypes.byref(h), ctypes.byref(d), None,
                            ofno.weight_count(**good)) == bvf.BVF_E_ARG
    assert L.bvf_fno_create(None, ctypes.byref(d), w, 4) == bvf.BVF_E_ARG
    assert L.bvf_fno_forward(None, 8, 8, 8, None, None, None) == bvf.BVF_E_ARG
    tab = bvf.material_array([(1000.0, 1500.0, 0, 0, 0, 0.6, 4180, 0, 0)])
    fake = ctypes.c_void_p(16)
    # k_src outside the grid, non-positive p_norm, bad material count: refused
    # before any device work
    assert L.bvf_fno_features(fake, tab, 1, tab, 8, 8, 8, 5e5, 8, fake, 1.0, fake,
                              None) == bvf.BVF_E_ARG
    assert L.bvf_fno_features(fake, tab, 1, tab, 8, 8, 8, 5e5, 0, fake, 0.0, fake,
                              None) == bvf.BVF_E_ARG
    assert L.bvf_fno_features(fake, tab, 0, tab, 8, 8, 8, 5e5, 0, fake, 1.0, fake,
                              None) == bvf.BVF_E_ARG
    L.bvf_fno_destroy(None)

