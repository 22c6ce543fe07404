"""The C-ABI library loads and exports every entry point include/bvf.h and
include/bvf_fno.h declare; host-side validation answers without touching a
GPU."""
import ctypes
import os
import re

import numpy as np

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
    assert bvf.bvf_version() == 3
    assert bvf.bvf_courant_limit() == pytest.approx(6 / (7 * 3 ** 0.5), rel=1e-15)
    assert bvf.lib().bvf_strerror(-2).decode().startswith("time step")
    assert bvf.lib().bvf_strerror(bvf.BVF_E_TIMEOUT).decode().startswith("wall-clock")


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
    assert L.bvf_set_time_budget(None, 1.0) == bvf.BVF_E_ARG
    assert L.bvf_state_bytes(None, None) == bvf.BVF_E_ARG
    assert L.bvf_state_save(None, None, 0, None) == bvf.BVF_E_ARG
    assert L.bvf_state_load(None, None, 0, None) == bvf.BVF_E_ARG
    assert L.bvf_test_withhold_copy(None, 1, 0, 0) == bvf.BVF_E_ARG
    assert L.bvf_time_reversal_plane(None, 0, 0, 0, 0, 10, 1500.0, None, None) == bvf.BVF_E_ARG
    assert L.bvf_steer_weights(None, 1, None, 5e5, 1500.0) == bvf.BVF_E_ARG
    t = bvf.Tile(8, 16, 0)
    assert L.bvf_set_tile(None, ctypes.byref(t)) == bvf.BVF_E_ARG
    assert L.bvf_get_tile(None, ctypes.byref(t)) == bvf.BVF_E_ARG
    assert L.bvf_batch_tune_domains(None, 1, ctypes.byref(t), 1, None, None) == bvf.BVF_E_ARG
    assert L.bvf_batch_tune_graph(None, 1, ctypes.byref(t), 1, 8, ctypes.byref(t), None,
                                  None) == bvf.BVF_E_ARG
    assert L.bvf_plan_host(None, None, None, None, 0, None, None, 0, None, None, None, None,
                           None, None, None) == bvf.BVF_E_ARG
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



# ---- host-only phased-source helpers (no GPU): pinned to cap geometry and to
# the in-phase arrival that defines steering

def test_bowl_array_lies_on_the_cap_and_tiles_its_area(bvf):
    """Every element sits on the sphere of radius roc about the centre of
    curvature (apex + roc * axis), inside the aperture, and the element areas
    add up to the cap area 2 pi R^2 (1 - cos theta_max), for a tilted axis."""
    a_d, R = 24e-3, 22e-3
    apex = np.array([1e-3, -2e-3, 3e-3])
    u = np.array([0.3, -0.2, 1.0])
    u /= np.linalg.norm(u)
    bowl = bvf.Bowl(a_d, R, tuple(apex), tuple(u), 0.0, 1500.0, 0.0)
    el = bvf.bvf_bowl_array(bowl, 7, 6)
    assert el.shape == (6 * 7 * 8 // 2, 6)
    centre = apex + R * u
    np.testing.assert_allclose(np.linalg.norm(el[:, :3] - centre, axis=1), R, rtol=1e-12)
    # polar angle of each element about the axis, seen from the centre
    cosang = ((centre - el[:, :3]) @ u) / R
    thmax = np.arcsin(0.5 * a_d / R)
    assert (cosang >= np.cos(thmax) - 1e-12).all()
    np.testing.assert_allclose(el[:, 3].sum(), 2 * np.pi * R * R * (1 - np.cos(thmax)), rtol=1e-12)
    assert (el[:, 4] == 1.0).all() and (el[:, 5] == 0.0).all()
    # counting call
    n = ctypes.c_int()
    assert bvf.lib().bvf_bowl_array(ctypes.byref(bowl), 7, 6, None, ctypes.byref(n)) == 0
    assert n.value == el.shape[0]
    assert bvf.lib().bvf_bowl_array(ctypes.byref(bowl), 0, 6, None, ctypes.byref(n)) == bvf.BVF_E_ARG


def test_steer_weights_bring_every_element_in_phase_at_the_target(bvf):
    """With w_e from bvf_steer_weights, every element's monochromatic wave
    w_e exp(-i k r_e) / r_e reaches the target with zero phase, so the coherent
    sum there equals sum 1/r_e (its largest possible magnitude); other points
    see less."""
    rng = np.random.default_rng(4)
    el = np.column_stack([rng.uniform(-0.01, 0.01, 50), rng.uniform(-0.01, 0.01, 50),
                          rng.uniform(-0.03, -0.02, 50), np.ones(50), np.ones(50), np.zeros(50)])
    f0, c0 = 5e5, 1500.0
    k = 2 * np.pi * f0 / c0
    tgt = np.array([2e-3, -1e-3, 0.01])
    st = bvf.bvf_steer_weights(el, tgt, f0, c0)
    assert st.shape == el.shape and np.array_equal(st[:, :4], el[:, :4])
    w = st[:, 4] + 1j * st[:, 5]
    np.testing.assert_allclose(np.abs(w), 1.0, rtol=1e-14)

    def field(x):
        r = np.linalg.norm(st[:, :3] - x, axis=1)
        return np.sum(w * np.exp(-1j * k * r) / r), np.sum(1.0 / r)

    p, bound = field(tgt)
    assert abs(p - bound) < 1e-10 * bound
    p2, bound2 = field(tgt + np.array([1.5e-3, 0.0, 0.0]))
    assert abs(p2) < 0.9 * bound2
