"""Multi-element phased sources: the weighted-element Rayleigh field against
the oracle, geometric steering in water (the steered field against the
oracle's FDTD, and the focus position), and time reversal (the conjugated
plane against the oracle's own point-source capture, and refocusing through a
skull phantom)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available()
    from paper_2301_12727_gb300 import build
    build.build()
    from paper_2301_12727_gb300 import bvf, phased, synth
    return bvf, phased, synth


def test_gpu_rs_elements_matches_oracle(mods, orc):
    bvf, phased, synth = mods
    rng = np.random.default_rng(21)
    ne = 300
    el = np.column_stack([rng.uniform(0, 0.02, ne), rng.uniform(0, 0.02, ne),
                          rng.uniform(-0.02, -0.005, ne), rng.uniform(1e-6, 4e-6, ne),
                          rng.standard_normal(ne), rng.standard_normal(ne)])
    nx, ny, dx, zp, f0 = 45, 38, 0.5e-3, 0.004, 5e5
    got = bvf.bvf_rs_elements(el, 1e4, 1500.0, nx, ny, dx, zp, f0).cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    ref = orc.rs_elements(el, 1e4, 1500.0, nx, ny, dx, zp, f0)
    assert np.abs(got - ref).max() < 5e-5 * np.abs(ref).max()


def argmax3(a):
    return np.array(np.unravel_index(np.argmax(a), a.shape))


def test_gpu_steered_array_focuses_off_axis_in_water(mods):
    """A 168-element cap (geometric focus on the axis at cell 32) steered 4.25 mm
    sideways in its focal plane: in water the FDTD amplitude maximum moves to
    within one cell of the target laterally, at the depth of the unsteered
    beam's maximum (within two cells; at this Fresnel number, about 2, that
    maximum lies short of the geometric focus)."""
    bvf, phased, synth = mods
    nx = ny = 64
    nz, dx, f0, n_pml = 64, 0.5e-3, 5e5, 6
    k_src = n_pml + 2
    dt, M = synth.choose_dt(dx, 1500.0, f0)
    apex = (31.5 * dx, 31.5 * dx, 32 * dx - 22e-3)
    base = phased.bowl_array(24e-3, 22e-3, apex, n_rings=7)
    tgt_ijk = (40, 32, 32)                      # (i, j, k)
    peaks = []
    for el in (base, phased.steer(base, np.array(tgt_ijk, dtype=np.float64) * dx, f0)):
        s = bvf.Solver(nx, ny, nz, dx, dt, f0, n_sls=0, n_pml=n_pml)
        s.set_materials(np.zeros((nz, ny, nx), np.uint8), [synth.water_row(f0)])
        plane = bvf.bvf_rs_elements(el, 1e4, 1500.0, nx, ny, dx, k_src * dx, f0)
        s.set_source(plane, k_src, 1500.0, bvf.BVF_ENV_RAMP_CW)
        n = int(1.3 * nz * dx / 1500.0 / dt) + 4 * M
        s.run(n, dft_start=n - 2 * M + 1, dft_steps=2 * M)
        s.synchronize()
        amp = s.amp_phase()[0].cpu().numpy()
        amp[: k_src + 6] = 0.0
        peaks.append(argmax3(amp)[::-1])        # (i, j, k)
        s.close()
    plain, steered = peaks
    assert abs(plain[0] - 31.5) <= 1 and abs(plain[1] - 31.5) <= 1      # on the axis
    assert abs(steered[0] - tgt_ijk[0]) <= 1 and abs(steered[1] - tgt_ijk[1]) <= 1
    assert abs(steered[2] - plain[2]) <= 2, (plain, steered)


def test_gpu_time_reversal_refocuses_through_the_skull(mods):
    """Phase conjugation of a point source at a target beyond the skull
    phantom: driving the source plane with the conjugated field puts the
    steady-state amplitude maximum behind the skull within 2 cells of the
    target."""
    bvf, phased, synth = mods
    c = synth.skull_case(64, 64, 56, dx=0.5e-3, n_steps=10, aperture=24e-3, roc=22e-3,
                         n_pml=6, seed=5)
    s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
    s.set_materials(c.index, c.materials)
    tgt = (36, 30, 46)
    M = c.steps_per_period
    n = int(1.5 * c.nz * c.dx / 1500.0 / c.dt) + 4 * M
    plane = phased.time_reversal_plane(s, tgt, c.k_src, n)
    s.set_source(1e4 * plane, c.k_src, 1500.0, bvf.BVF_ENV_RAMP_CW)
    s.run(n, dft_start=n - 2 * M + 1, dft_steps=2 * M)
    s.synchronize()
    amp = s.amp_phase()[0].cpu().numpy()
    beyond = (c.index == 1)                     # brain, behind the skull
    got = argmax3(np.where(beyond, amp, 0.0))[::-1]
    assert np.abs(got - np.array(tgt)).max() <= 2, got
    s.close()


def test_gpu_time_reversal_plane_matches_oracle(mods, orc):
    """bvf_time_reversal_plane against the oracle: the same CW point source
    (one-cycle ramp) at the target behind a small skull phantom, run in FP64;
    its complex amplitude on the source plane over the last two periods,
    conjugated and divided by its largest magnitude, equals the library's
    plane to 2e-4 of that largest magnitude (FP32 fields over ~300 steps)."""
    bvf, phased, synth = mods
    c = synth.skull_case(48, 48, 40, dx=0.5e-3, n_steps=10, aperture=20e-3, roc=18e-3,
                         n_pml=4, seed=9)
    s = bvf.Solver(c.nx, c.ny, c.nz, c.dx, c.dt, c.f0, n_sls=2, n_pml=c.n_pml)
    s.set_materials(c.index, c.materials)
    tgt = (27, 21, 33)
    M = c.steps_per_period
    n = int(1.2 * c.nz * c.dx / 1500.0 / c.dt) + 3 * M
    got = phased.time_reversal_plane(s, tgt, c.k_src, n).cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    st = s.stats()
    assert st.steps == 0                       # reset afterwards
    s.close()
    A = orc.Acoustic(c.nx, c.ny, c.nz, c.dx, c.dt, c.index, c.materials, c.f0, n_sls=2,
                     n_pml=c.n_pml)
    pt = np.zeros((c.ny, c.nx), dtype=np.complex128)
    pt[tgt[1], tgt[0]] = 1.0
    A.set_source(pt, tgt[2], 1500.0, orc.ENV_RAMP_CW)
    assert A.run(n, peak_from=-1, dft_start=n - 2 * M + 1, dft_steps=2 * M) == 0
    amp, ph = A.amp_phase(2 * M)
    P = amp[c.k_src] * np.exp(1j * ph[c.k_src])
    ref = np.conj(P) / np.abs(P).max()
    assert np.abs(got).max() == pytest.approx(1.0, abs=1e-6)
    assert np.abs(got - ref).max() < 2e-4


def test_gpu_steered_field_matches_oracle(mods, orc):
    """A steered 84-element cap in water: the library's weighted Rayleigh plane
    and FDTD amplitude against the oracle's Rayleigh plane and FP64 FDTD with
    the same weights (relative L2 of the amplitude < 1e-4)."""
    bvf, phased, synth = mods
    nx = ny = 48
    nz, dx, f0, n_pml = 40, 0.5e-3, 5e5, 4
    k_src = n_pml + 2
    dt, M = synth.choose_dt(dx, 1500.0, f0)
    apex = (23.5 * dx, 23.5 * dx, k_src * dx - 5e-3)
    base = phased.bowl_array(16e-3, 16e-3, apex, n_rings=6, n_inner=4)
    el = phased.steer(base, np.array([28.0, 21.0, 26.0]) * dx, f0)
    plane = bvf.bvf_rs_elements(el, 1e4, 1500.0, nx, ny, dx, k_src * dx, f0)
    s = bvf.Solver(nx, ny, nz, dx, dt, f0, n_sls=0, n_pml=n_pml)
    idx = np.zeros((nz, ny, nx), np.uint8)
    s.set_materials(idx, [synth.water_row(f0)])
    s.set_source(plane, k_src, 1500.0, bvf.BVF_ENV_RAMP_CW)
    n = int(1.2 * nz * dx / 1500.0 / dt) + 3 * M
    s.run(n, dft_start=n - 2 * M + 1, dft_steps=2 * M)
    s.synchronize()
    amp = s.amp_phase()[0].cpu().numpy()
    s.close()
    ref_plane = orc.rs_elements(el, 1e4, 1500.0, nx, ny, dx, k_src * dx, f0)
    A = orc.Acoustic(nx, ny, nz, dx, dt, idx, [synth.water_row(f0)], f0, n_sls=0, n_pml=n_pml)
    A.set_source(ref_plane, k_src, 1500.0, orc.ENV_RAMP_CW)
    assert A.run(n, peak_from=-1, dft_start=n - 2 * M + 1, dft_steps=2 * M) == 0
    ref = A.amp_phase(2 * M)[0]
    assert np.linalg.norm(amp - ref) / np.linalg.norm(ref) < 1e-4
